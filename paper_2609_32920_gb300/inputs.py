"""Seeded synthetic scene generators.

This module only builds input data (geometry arrays, textures, heights, camera
parameters, adjoint images).  It contains none of the light-tracing arithmetic,
so both the CUDA path and the CPU oracle can consume its output without sharing
any of the method's code.

Scene layout (all float64 / int32 numpy arrays):

* ``quads``     [nq, 9]  analytic parallelograms ``o, e1, e2`` (point = o + s e1 + t e2,
  s, t in [0, 1]); primitive ids ``0 .. nq-1``.
* ``verts``     [nv, 3]  triangle vertex base positions.
* ``vert_h``    [nv]     index of the height parameter added to the vertex y, or -1.
* ``tris``      [nt, 3]  vertex indices; primitive ids ``nq .. nq+nt-1``.  The geometric
  normal is ``cross(v1 - v0, v2 - v0)``.
* ``prim_mat``  [nq+nt]  material id per primitive.
* ``mat_type``  [nm]     0 diffuse (textured), 1 smooth dielectric, 2 emitter.
* ``mat_ior``   [nm]     index of refraction (dielectric only).
* ``mat_tex_off/w/h`` [nm] texel offset (in floats) into the albedo parameter array and
  the texture size; a diffuse material's texture is ``h x w x 3`` (row-major, RGB).
* ``emitter_quad``       quad index of the (one-sided) area emitter; it emits along
  ``cross(e1, e2)``.
* camera: ``cam_pos``, ``cam_look``, ``cam_up``, ``fov_y_deg``, ``W``, ``H``.
* parameters: ``albedo`` [n_albedo], ``Le`` [3], ``heights`` [n_h].

The generators below build the synthetic workloads: the textured box, the box with a
diffuse height field, the dielectric caustic slab, the batched set of uneven scenes and
the scenes of the learned-target study, each fully determined by its arguments and seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DIFFUSE, DIELECTRIC, EMITTER = 0, 1, 2


@dataclass
class Scene:
    quads: np.ndarray
    verts: np.ndarray
    vert_h: np.ndarray
    tris: np.ndarray
    prim_mat: np.ndarray
    mat_type: np.ndarray
    mat_ior: np.ndarray
    mat_tex_off: np.ndarray
    mat_tex_w: np.ndarray
    mat_tex_h: np.ndarray
    emitter_quad: int
    cam_pos: np.ndarray
    cam_look: np.ndarray
    cam_up: np.ndarray
    fov_y_deg: float
    W: int
    H: int
    albedo: np.ndarray
    Le: np.ndarray
    heights: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_quads(self) -> int:
        return int(self.quads.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_prims(self) -> int:
        return self.n_quads + self.n_tris

    def with_params(self, albedo=None, Le=None, heights=None) -> "Scene":
        import copy
        s = copy.copy(self)
        if albedo is not None:
            s.albedo = np.ascontiguousarray(albedo, dtype=np.float64)
        if Le is not None:
            s.Le = np.ascontiguousarray(Le, dtype=np.float64)
        if heights is not None:
            s.heights = np.ascontiguousarray(heights, dtype=np.float64)
        return s


class _Builder:
    def __init__(self):
        self.quads: list = []
        self.quad_mat: list = []
        self.verts: list = []
        self.vert_h: list = []
        self.tris: list = []
        self.tri_mat: list = []
        self.mat_type: list = []
        self.mat_ior: list = []
        self.mat_tex_off: list = []
        self.mat_tex_w: list = []
        self.mat_tex_h: list = []
        self.albedo: list = []
        self.n_albedo = 0
        self.n_heights = 0
        self.emitter_quad = -1

    def diffuse(self, tex: np.ndarray) -> int:
        tex = np.asarray(tex, dtype=np.float64)
        assert tex.ndim == 3 and tex.shape[2] == 3
        m = len(self.mat_type)
        self.mat_type.append(DIFFUSE)
        self.mat_ior.append(1.0)
        self.mat_tex_off.append(self.n_albedo)
        self.mat_tex_h.append(tex.shape[0])
        self.mat_tex_w.append(tex.shape[1])
        self.albedo.append(tex.reshape(-1))
        self.n_albedo += tex.size
        return m

    def dielectric(self, ior: float) -> int:
        m = len(self.mat_type)
        self.mat_type.append(DIELECTRIC)
        self.mat_ior.append(float(ior))
        self.mat_tex_off.append(0)
        self.mat_tex_w.append(0)
        self.mat_tex_h.append(0)
        return m

    def emitter(self) -> int:
        m = len(self.mat_type)
        self.mat_type.append(EMITTER)
        self.mat_ior.append(1.0)
        self.mat_tex_off.append(0)
        self.mat_tex_w.append(0)
        self.mat_tex_h.append(0)
        return m

    def quad(self, o, e1, e2, mat: int) -> int:
        self.quads.append(np.concatenate([o, e1, e2]).astype(np.float64))
        self.quad_mat.append(mat)
        return len(self.quads) - 1

    def vertex(self, p, h_index: int = -1) -> int:
        self.verts.append(np.asarray(p, dtype=np.float64))
        self.vert_h.append(h_index)
        return len(self.verts) - 1

    def tri(self, a: int, b: int, c: int, mat: int):
        self.tris.append((a, b, c))
        self.tri_mat.append(mat)

    def heightmap(self, nx: int, nz: int, x0: float, z0: float, ex: float, ez: float,
                  y0: float, mat: int, flip: bool = False) -> np.ndarray:
        """Grid of nx*nz vertices on y=y0 + h[j, i]; 2 (nx-1)(nz-1) triangles with +y normals
        (or -y when ``flip``).  Returns the vertex index grid [nz, nx]."""
        base_h = self.n_heights
        self.n_heights += nx * nz
        idx = np.zeros((nz, nx), dtype=np.int64)
        for j in range(nz):
            for i in range(nx):
                p = (x0 + ex * i / (nx - 1), y0, z0 + ez * j / (nz - 1))
                idx[j, i] = self.vertex(p, base_h + j * nx + i)
        for j in range(nz - 1):
            for i in range(nx - 1):
                v00, v10 = idx[j, i], idx[j, i + 1]
                v01, v11 = idx[j + 1, i], idx[j + 1, i + 1]
                if not flip:
                    self.tri(v00, v11, v10, mat)
                    self.tri(v00, v01, v11, mat)
                else:
                    self.tri(v00, v10, v11, mat)
                    self.tri(v00, v11, v01, mat)
        return idx

    def build(self, cam_pos, cam_look, cam_up, fov_y_deg, W, H, Le, heights, name, meta=None) -> Scene:
        assert self.emitter_quad >= 0
        prim_mat = np.array(self.quad_mat + self.tri_mat, dtype=np.int32)
        return Scene(
            quads=np.array(self.quads, dtype=np.float64).reshape(-1, 9),
            verts=np.array(self.verts, dtype=np.float64).reshape(-1, 3),
            vert_h=np.array(self.vert_h, dtype=np.int32),
            tris=np.array(self.tris, dtype=np.int32).reshape(-1, 3),
            prim_mat=prim_mat,
            mat_type=np.array(self.mat_type, dtype=np.int32),
            mat_ior=np.array(self.mat_ior, dtype=np.float64),
            mat_tex_off=np.array(self.mat_tex_off, dtype=np.int32),
            mat_tex_w=np.array(self.mat_tex_w, dtype=np.int32),
            mat_tex_h=np.array(self.mat_tex_h, dtype=np.int32),
            emitter_quad=int(self.emitter_quad),
            cam_pos=np.asarray(cam_pos, dtype=np.float64),
            cam_look=np.asarray(cam_look, dtype=np.float64),
            cam_up=np.asarray(cam_up, dtype=np.float64),
            fov_y_deg=float(fov_y_deg), W=int(W), H=int(H),
            albedo=(np.concatenate(self.albedo) if self.albedo else np.zeros(0)).astype(np.float64),
            Le=np.asarray(Le, dtype=np.float64),
            heights=np.asarray(heights, dtype=np.float64).reshape(-1),
            name=name, meta=dict(meta or {}),
        )


def _torch_uniform(shape, lo, hi, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    return (lo + (hi - lo) * torch.rand(shape, generator=g, dtype=torch.float64)).numpy()


def _torch_normal(shape, std, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    return (std * torch.randn(shape, generator=g, dtype=torch.float64)).numpy()


def _box_walls(b: _Builder, textures):
    """The open box [0,1]^3 (face z=0 missing): floor, ceiling, back, left, right."""
    walls = [
        ((0, 0, 0), (0, 0, 1), (1, 0, 0)),   # floor    y=0, normal +y
        ((0, 1, 0), (1, 0, 0), (0, 0, 1)),   # ceiling  y=1, normal -y
        ((0, 0, 1), (0, 1, 0), (1, 0, 0)),   # back     z=1, normal -z
        ((0, 0, 0), (0, 1, 0), (0, 0, 1)),   # left     x=0, normal +x
        ((1, 0, 0), (0, 0, 1), (0, 1, 0)),   # right    x=1, normal -x
    ]
    for (o, e1, e2), tex in zip(walls, textures):
        m = b.diffuse(tex)
        b.quad(np.array(o, float), np.array(e1, float), np.array(e2, float), m)


def _box_light(b: _Builder, size=0.25, y=0.99):
    m = b.emitter()
    o = np.array([0.5 - size / 2, y, 0.5 - size / 2])
    b.emitter_quad = b.quad(o, np.array([size, 0, 0.0]), np.array([0, 0, size]), m)  # normal -y


def box_scene(res: int = 64, tex_seed: int = 0, tex_size: int = 16, Le=(8.0, 8.0, 8.0),
              heightmap: int = 0, hm_seed: int = 0, hm_std: float = 0.02) -> Scene:
    """Cornell-style open box; optional ``heightmap x heightmap`` diffuse plane at y=0.25
    over x,z in [0.25, 0.75] with heights N(0, hm_std) (seeded)."""
    b = _Builder()
    tex = _torch_uniform((5, tex_size, tex_size, 3), 0.2, 0.8, tex_seed)
    _box_walls(b, list(tex))
    _box_light(b)
    heights = np.zeros(0)
    if heightmap:
        m = b.diffuse(np.full((1, 1, 3), 0.5))
        b.heightmap(heightmap, heightmap, 0.25, 0.25, 0.5, 0.5, 0.25, m)
        heights = _torch_normal((heightmap * heightmap,), hm_std, hm_seed)
    name = f"box{res}" + (f"_hm{heightmap}" if heightmap else "")
    return b.build((0.5, 0.5, -1.4), (0.5, 0.5, 0.0), (0, 1, 0), 40.0, res, res, Le, heights, name,
                   meta={"kind": "box", "heightmap": heightmap})


def gaussian_bumps(n: int, extent: float, seed: int, n_gauss: int = 8, amp_std: float = 0.01):
    """Heights on an n x n grid spanning [-extent/2, extent/2]^2: sum of ``n_gauss`` Gaussians
    with amplitudes N(0, amp_std), centres uniform over the grid, sigma U[0.05, 0.2]."""
    import torch
    g = torch.Generator().manual_seed(seed)
    amp = (amp_std * torch.randn(n_gauss, generator=g, dtype=torch.float64)).numpy()
    cen = ((torch.rand(n_gauss, 2, generator=g, dtype=torch.float64) - 0.5) * extent).numpy()
    sig = (0.05 + 0.15 * torch.rand(n_gauss, generator=g, dtype=torch.float64)).numpy()
    xs = np.linspace(-extent / 2, extent / 2, n)
    X, Z = np.meshgrid(xs, xs)  # [z, x]
    h = np.zeros((n, n))
    for a, (cx, cz), s in zip(amp, cen, sig):
        h += a * np.exp(-((X - cx) ** 2 + (Z - cz) ** 2) / (2 * s * s))
    return h.reshape(-1)


def _slab(b: _Builder, n: int, x0: float, z0: float, size: float, y_bottom: float, y_top: float, ior: float):
    """A dielectric slab over [x0, x0+size] x [z0, z0+size]: an n x n height-field top at
    y_top, a flat bottom at y_bottom, and side strips that follow the top's boundary
    heights (bottom edge fixed)."""
    gm = b.dielectric(ior)
    top = b.heightmap(n, n, x0, z0, size, size, y_top, gm)
    # bottom face (normal -y): two triangles on fixed vertices
    x1, z1 = x0 + size, z0 + size
    c = [b.vertex((x0, y_bottom, z0)), b.vertex((x1, y_bottom, z0)),
         b.vertex((x1, y_bottom, z1)), b.vertex((x0, y_bottom, z1))]
    b.tri(c[0], c[1], c[2], gm)
    b.tri(c[0], c[2], c[3], gm)
    # side strips: bottom edge fixed at y_bottom, top edge = heightmap boundary vertices

    def strip(top_line, bot_a, bot_b, outward):
        # top_line: vertex indices along the edge; bottom edge interpolated with fixed verts
        k = len(top_line)
        bot = [bot_a] + [b.vertex(tuple(b.verts[bot_a] + (b.verts[bot_b] - b.verts[bot_a]) * (i / (k - 1))))
                         for i in range(1, k - 1)] + [bot_b]
        for i in range(k - 1):
            t0, t1, b0, b1 = top_line[i], top_line[i + 1], bot[i], bot[i + 1]
            # orient so that cross(v1-v0, v2-v0) points along `outward`
            p0, p1, p2 = b.verts[b0], b.verts[b1], b.verts[t1]
            nrm = np.cross(p1 - p0, p2 - p0)
            if np.dot(nrm, outward) > 0:
                b.tri(b0, b1, t1, gm)
                b.tri(b0, t1, t0, gm)
            else:
                b.tri(b0, t1, b1, gm)
                b.tri(b0, t0, t1, gm)
    strip(list(top[0, :]), c[0], c[1], np.array([0, 0, -1.0]))      # z = z0
    strip(list(top[n - 1, :]), c[3], c[2], np.array([0, 0, 1.0]))   # z = z0 + size
    strip(list(top[:, 0]), c[0], c[3], np.array([-1.0, 0, 0]))      # x = x0
    strip(list(top[:, n - 1]), c[1], c[2], np.array([1.0, 0, 0]))   # x = x0 + size


def slab_scene(res: int = 512, n: int = 128, seed: int = 0, Le_scale: float = 1.0,
               light_size: float = 0.05, ior: float = 1.5, flat: bool = False) -> Scene:
    """Caustic workload: 2x2 m diffuse receiver (albedo 0.7) at y=0, a 1x1 m dielectric slab
    with flat bottom at y=0.5 and an n x n heightmap top at y=0.6 (sum of Gaussians), sides
    closed by strips that follow the boundary heights, small light at y=2.0 facing -y."""
    b = _Builder()
    rm = b.diffuse(np.full((1, 1, 3), 0.7))
    b.quad(np.array([-1.0, 0, -1.0]), np.array([0, 0, 2.0]), np.array([2.0, 0, 0]), rm)  # +y
    em = b.emitter()
    ls = light_size
    b.emitter_quad = b.quad(np.array([-ls / 2, 2.0, -ls / 2]), np.array([ls, 0, 0.0]),
                            np.array([0, 0, ls]), em)  # -y
    _slab(b, n, -0.5, -0.5, 1.0, 0.5, 0.6, ior)
    heights = np.zeros(n * n) if flat else gaussian_bumps(n, 1.0, seed)
    # Le chosen so that the mean receiver pixel is O(1) for the default camera
    Le = np.full(3, 2000.0 * Le_scale)
    return b.build((0.0, 1.2, -1.6), (0.0, 0.0, 0.0), (0, 1, 0), 45.0, res, res, Le, heights,
                   f"slab{res}_hm{n}", meta={"kind": "slab", "heightmap": n})


def slab_in_box(res: int = 256, n: int = 64, seed: int = 0, tex_seed: int = 0, ior: float = 1.5) -> Scene:
    """The caustic slab inside the textured box (high path-sensor connectivity with
    refraction): the open box of box_scene with its emitter, and a 0.5 x 0.5 m dielectric
    slab over x, z in [0.25, 0.75], flat bottom at y=0.2, n x n height-field top at y=0.3
    (sum of Gaussians, amplitudes N(0, 0.005) m)."""
    b = _Builder()
    tex = _torch_uniform((5, 16, 16, 3), 0.2, 0.8, tex_seed)
    _box_walls(b, list(tex))
    _box_light(b)
    _slab(b, n, 0.25, 0.25, 0.5, 0.2, 0.3, ior)
    heights = gaussian_bumps(n, 0.5, seed, amp_std=0.005)
    return b.build((0.5, 0.5, -1.4), (0.5, 0.5, 0.0), (0, 1, 0), 40.0, res, res, (8.0, 8.0, 8.0), heights,
                   f"slabbox{res}_hm{n}", meta={"kind": "slab_in_box", "heightmap": n})


def plane_under_light(res: int = 32, albedo: float = 0.5, light_size: float = 0.5, light_h: float = 1.0,
                      Le=(1.0, 1.0, 1.0), heightmap: int = 0, hm_std: float = 0.0, hm_seed: int = 0,
                      plane_half: float = 2.0) -> Scene:
    """Closed-form workload: a large diffuse plane y=0 (uniform albedo) under a square
    one-sided emitter parallel to it at height ``light_h``; camera straight above looking
    down through the (one-sided, back-face black) emitter's side.  With ``heightmap`` the
    central plane is a small diffuse height field instead (for smooth attached tests)."""
    b = _Builder()
    m = b.diffuse(np.full((1, 1, 3), albedo))
    if heightmap:
        b.heightmap(heightmap, heightmap, -plane_half, -plane_half, 2 * plane_half, 2 * plane_half, 0.0, m)
    else:
        b.quad(np.array([-plane_half, 0, -plane_half]), np.array([0, 0, 2 * plane_half]),
               np.array([2 * plane_half, 0, 0]), m)
    em = b.emitter()
    s = light_size
    b.emitter_quad = b.quad(np.array([-s / 2, light_h, -s / 2]), np.array([s, 0, 0.0]),
                            np.array([0, 0, s]), em)
    heights = np.zeros(heightmap * heightmap)
    if heightmap and hm_std > 0:
        heights = _torch_normal((heightmap * heightmap,), hm_std, hm_seed)
    # camera to the side and above, looking at the lit region
    return b.build((1.6, 1.3, 0.0), (0.3, 0.0, 0.0), (0, 1, 0), 40.0, res, res, Le, heights,
                   "plane_under_light", meta={"kind": "plane", "light_size": s, "light_h": light_h,
                                              "albedo": albedo, "heightmap": heightmap})


def smooth_adjoint(W: int, H: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A fixed, smooth, signed image-space adjoint dL/dI [H, W, 3] (float64)."""
    import torch
    g = torch.Generator().manual_seed(seed)
    coarse = torch.randn(1, 3, max(2, H // 8), max(2, W // 8), generator=g, dtype=torch.float64)
    fine = torch.nn.functional.interpolate(coarse, size=(H, W), mode="bilinear", align_corners=False)
    noise = 0.25 * torch.randn(1, 3, H, W, generator=g, dtype=torch.float64)
    a = (fine + noise)[0].permute(1, 2, 0).contiguous().numpy()
    return scale * a / (W * H)


def blob_adjoint(W: int, H: int, seed: int, sigma: float = 0.12, scale: float = 1.0) -> np.ndarray:
    """A spatially concentrated signed adjoint [H, W, 3]: a Gaussian blob at a seeded film
    position (the image difference of an inverse problem that is wrong in one region) plus
    10% smooth background."""
    import torch
    g = torch.Generator().manual_seed(seed)
    cx, cy = (0.25 + 0.5 * torch.rand(2, generator=g, dtype=torch.float64)).tolist()
    sgn = (torch.rand(3, generator=g, dtype=torch.float64) * 0.5 + 0.75).numpy()
    ys, xs = np.meshgrid((np.arange(H) + 0.5) / H, (np.arange(W) + 0.5) / W, indexing="ij")
    blob = np.exp(-((xs - cx) ** 2 + (ys - cy) ** 2) / (2 * sigma * sigma))
    a = blob[..., None] * sgn[None, None, :] + 0.1 * smooth_adjoint(W, H, seed + 1) * (W * H)
    return scale * a / (W * H)


def perturbed_albedo(scene: Scene, std: float = 0.05, seed: int = 1) -> np.ndarray:
    """Target albedo: albedo + N(0, std), clamped to [0.05, 0.95]."""
    n = _torch_normal(scene.albedo.shape, std, seed)
    return np.clip(scene.albedo + n, 0.05, 0.95)


# ------------------------------------------------------------------ named workloads
def workload(name: str) -> dict:
    """Named workload presets.  Returns dict(scene=..., n_paths=..., max_depth=..., attached=...)."""
    if name == "box64":          # 64x64 box, depth 4, 2^14 paths, detached albedo
        return dict(scene=box_scene(64), n_paths=1 << 14, max_depth=4, attached=0)
    if name == "box256_hm32":    # 256x256 box + 32x32 heightmap, depth 16, 2^22 paths, attached
        return dict(scene=box_scene(256, heightmap=32), n_paths=1 << 22, max_depth=16, attached=1)
    if name == "slab512_hm128":  # caustic slab, 512x512, depth 8, 2^24 paths, attached
        return dict(scene=slab_scene(512, 128), n_paths=1 << 24, max_depth=8, attached=1)
    raise KeyError(name)


def batched_set(n_scenes: int = 64, seed: int = 0, max_paths_log2: int = 22):
    """Uneven batch: heightmap side round(2^U[5,8]), depth U{4..32}, paths 2^round(U[16,22]),
    alternating slab / box type, all seeded by scene id."""
    import torch
    g = torch.Generator().manual_seed(seed)
    out = []
    for i in range(n_scenes):
        side = int(round(2 ** (5 + 3 * torch.rand(1, generator=g).item())))
        depth = int(4 + torch.randint(0, 29, (1,), generator=g).item())
        lp = int(round(16 + (max_paths_log2 - 16) * torch.rand(1, generator=g).item()))
        if i % 2 == 0:
            sc = slab_scene(128, n=side, seed=i)
        else:
            sc = box_scene(128, heightmap=side, hm_seed=i)
        out.append(dict(scene=sc, n_paths=1 << lp, max_depth=depth, attached=1))
    return out
