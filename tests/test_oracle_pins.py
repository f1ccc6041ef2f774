"""Pins of the FP64 CPU oracle against things other than itself: closed forms,
reciprocity with a path tracer, finite differences, exact invariants, special cases
and statistical properties the paper states (CPU only)."""
import numpy as np
import pytest

from paper_2609_32920_gb300 import inputs as I


# ----------------------------------------------------------------------------- RNG
def test_philox_uniformity_and_avalanche(oracle):
    """Counter-based generator (Salmon et al. 2011): uniform words, independent counters,
    and each counter bit flips about half of the output bits."""
    n = 1 << 15
    words = np.array([oracle.philox((0x1234, 0x9876), (i, 0, 7, 0)) for i in range(n)], dtype=np.uint64)
    for w in range(4):
        hist = np.bincount((words[:, w] >> 26).astype(np.int64), minlength=64)
        chi2 = ((hist - n / 64) ** 2 / (n / 64)).sum()
        assert chi2 < 120, chi2  # 63 dof, p ~ 1e-5
        bits = np.unpackbits(words[:, w].astype(np.uint32).view(np.uint8)).reshape(n, 32).mean(0)
        assert np.all(np.abs(bits - 0.5) < 0.02)
    base = oracle.philox((5, 6), (1, 2, 3, 4)).astype(np.uint32)
    flips = []
    for word in range(4):
        for bit in range(32):
            c = [1, 2, 3, 4]
            c[word] ^= 1 << bit
            o = oracle.philox((5, 6), c).astype(np.uint32)
            flips.append(np.unpackbits((o ^ base).view(np.uint8)).sum())
    assert 56 < np.mean(flips) < 72  # of 128 bits
    # key changes the stream too
    assert not np.array_equal(oracle.philox((5, 7), (1, 2, 3, 4)), base)


def test_philox_known_answer_vectors(oracle):
    """The generator reproduces the published known-answer vectors of Philox4x32-10
    (tests/golden/philox4x32_10_kat.txt, Salmon et al. SC'11): counter, key -> four words."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox((v[4], v[5]), tuple(v[0:4])).astype(np.uint64)
        assert [int(x) for x in out] == v[6:10], (r, [hex(int(x)) for x in out])


def test_uniforms_exact_in_float32(oracle):
    """24-bit uniforms are exactly representable in fp32, so both precisions see the same numbers."""
    u = np.array([oracle.uniforms(99, i, d) for i in range(200) for d in range(3)]).ravel()
    assert np.all(u >= 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert np.array_equal(np.round(u * 2 ** 24), u * 2 ** 24)


# ----------------------------------------------------------------------- dielectric
def test_dielectric_fresnel_and_snell(oracle):
    n = np.array([0.0, 1.0, 0.0])
    # normal incidence: F = ((n1-n2)/(n1+n2))^2
    d, F, refl = oracle.dielectric([0, -1.0, 0], n, 1.5, 0.9)
    assert F == pytest.approx(0.04, abs=1e-12) and not refl
    assert np.allclose(d, [0, -1, 0])
    rng = np.random.default_rng(0)
    for _ in range(200):
        th = rng.uniform(0, np.pi / 2 * 0.99)
        phi = rng.uniform(0, 2 * np.pi)
        din = np.array([np.sin(th) * np.cos(phi), -np.cos(th), np.sin(th) * np.sin(phi)])
        out, F, refl = oracle.dielectric(din, n, 1.5, 1.0 - 1e-12)  # force refraction when possible
        assert not refl
        sin_t = np.linalg.norm(np.cross(out, n))
        assert sin_t == pytest.approx(np.sin(th) / 1.5, abs=1e-12)  # Snell
        assert np.linalg.norm(out) == pytest.approx(1.0, abs=1e-12)
        assert np.dot(np.cross(din, n), out) == pytest.approx(0.0, abs=1e-12)  # plane of incidence
        rl, F2, refl2 = oracle.dielectric(din, n, 1.5, 0.0)
        assert refl2 and np.allclose(rl, din - 2 * np.dot(din, n) * n)
    # Brewster angle: p-polarised reflectance vanishes, F = Rs/2
    tb = np.arctan(1.5)
    din = np.array([np.sin(tb), -np.cos(tb), 0])
    _, F, _ = oracle.dielectric(din, n, 1.5, 0.5)
    ct = np.sqrt(1 - (np.sin(tb) / 1.5) ** 2)
    rs = (np.cos(tb) - 1.5 * ct) / (np.cos(tb) + 1.5 * ct)
    assert F == pytest.approx(rs * rs / 2, rel=1e-10)
    # total internal reflection beyond the critical angle from inside
    tc = np.arcsin(1 / 1.5)
    for th in (tc + 0.01, 1.2):
        din = np.array([np.sin(th), np.cos(th), 0])  # travelling +y, exiting through normal +y
        out, F, refl = oracle.dielectric(din, n, 1.5, 0.999)
        assert refl and F == 1.0 and np.allclose(out, [np.sin(th), -np.cos(th), 0])
    # just below the critical angle the ray exits and bends away from the normal
    th = tc - 0.05
    out, F, refl = oracle.dielectric([np.sin(th), np.cos(th), 0], n, 1.5, 0.999)
    assert not refl and np.linalg.norm(np.cross(out, n)) == pytest.approx(1.5 * np.sin(th), abs=1e-12)


# ------------------------------------------------------------------------ reservoir
def test_reservoir_selection_pmf_and_unbiasedness(oracle):
    """Eq. 8: Pr(R=i) = w_i / Omega_k; Eq. 10: E[(Omega_k/w_R) x_R] = sum_i x_i."""
    rng = np.random.default_rng(1)
    w = np.array([0.3, 0.0, 1.7, 0.05, 0.9, 2.2])
    x = rng.normal(size=w.size)
    M = 40000
    counts = np.zeros(w.size)
    est = np.zeros(M)
    for m in range(M):
        R, rw = oracle.reservoir(w, rng.random(w.size))
        counts[R] += 1
        est[m] = rw * x[R]
        assert rw == pytest.approx(w.sum() / w[R])
    p = w / w.sum()
    nz = p > 0
    chi2 = ((counts[nz] - M * p[nz]) ** 2 / (M * p[nz])).sum()
    assert counts[~nz].sum() == 0
    assert chi2 < 25  # 4 dof
    assert abs(est.mean() - x[nz].sum()) < 4 * est.std() / np.sqrt(M)
    R, rw = oracle.reservoir(np.zeros(3), np.zeros(3))
    assert R == -1 and rw == 0


# ----------------------------------------------------------------------- primal image
def _lambert_polygon_irradiance(x, corners, Le):
    """Irradiance at x on a +y-facing plane from a Lambertian polygon (Lambert's formula)."""
    n = np.array([0, 1.0, 0])
    v = [(c - x) / np.linalg.norm(c - x) for c in corners]
    tot = 0.0
    for k in range(len(v)):
        a, b = v[k], v[(k + 1) % len(v)]
        cr = np.cross(a, b)
        tot += np.arccos(np.clip(a @ b, -1, 1)) * (n @ cr) / np.linalg.norm(cr)
    return abs(Le * tot / 2)


def test_primal_closed_form_area_light_over_plane(oracle):
    """Direct light (depth 1) on a diffuse plane under a square Lambertian emitter: pixel =
    tent-weighted average over the on-film footprint of rho E / pi, E from Lambert's formula."""
    sc = I.plane_under_light(res=16)
    rho = sc.meta["albedo"]
    q = sc.quads[sc.emitter_quad]
    o, e1, e2 = q[:3], q[3:6], q[6:9]
    corners = [o, o + e1, o + e1 + e2, o + e2]
    f = sc.cam_look - sc.cam_pos
    f /= np.linalg.norm(f)
    r = np.cross(f, sc.cam_up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    tany = np.tan(np.radians(sc.fov_y_deg) / 2)
    tanx = tany * sc.W / sc.H
    g = (np.arange(12) + 0.5) / 12 * 2 - 1
    tw = 1 - np.abs(g)
    tw /= tw.sum()
    ref = np.zeros((sc.H, sc.W))
    for py in range(sc.H):
        for px in range(sc.W):
            acc = 0.0
            for a, wa in zip(g, tw):
                for b, wb in zip(g, tw):
                    ux, uy = px + 0.5 + a, py + 0.5 + b
                    if not (0 <= ux < sc.W and 0 <= uy < sc.H):
                        continue  # the light tracer only splats connections landing on the film
                    d = f + r * (2 * ux / sc.W - 1) * tanx + u * (1 - 2 * uy / sc.H) * tany
                    x = sc.cam_pos + (-sc.cam_pos[1] / d[1]) * d
                    acc += wa * wb * rho * _lambert_polygon_irradiance(x, corners, 1.0) / np.pi
            ref[py, px] = acc
    B, N = 16, 1 << 17
    imgs = np.array([oracle.render(sc, seed=s, n_paths=N, max_depth=1)[..., 0] for s in range(B)])
    m = imgs.mean(0)
    se = imgs.std(0, ddof=1) / np.sqrt(B)
    z = (m - ref) / se
    assert np.mean(z ** 2) < 1.6
    assert np.mean(np.abs(z) > 3) < 0.03
    assert abs(m.sum() / ref.sum() - 1) < 4 * np.sqrt((se ** 2).sum()) / ref.sum()
    # the three channels are identical for a grey scene
    img = oracle.render(sc, seed=0, n_paths=1 << 12, max_depth=1)
    assert np.array_equal(img[..., 0], img[..., 1])


def test_primal_reciprocity_with_path_tracer(oracle):
    """Light tracing and camera-side path tracing estimate the same image (box with a
    diffuse height field, depth 3): per-pixel agreement within Monte Carlo error."""
    sc = I.box_scene(12, heightmap=4, hm_std=0.05)
    D, B = 3, 16
    lts = np.array([oracle.render(sc, seed=s, n_paths=1 << 17, max_depth=D) for s in range(B)])
    pts = np.array([oracle.render_pt(sc, seed=100 + s, spp=96, max_depth=D) for s in range(B)])
    se = np.sqrt(lts.var(0, ddof=1) / B + pts.var(0, ddof=1) / B)
    z = (lts.mean(0) - pts.mean(0)) / se
    assert np.mean(z ** 2) < 1.5
    assert np.mean(np.abs(z) > 3.5) < 0.02
    tot = lts.mean(0).sum() / pts.mean(0).sum()
    assert abs(tot - 1) < 0.01


# ------------------------------------------------------------------ gradients (exact)
def _loss_fd(oracle, sc, dI, p0, p1, **kw):
    return oracle.frozen_loss(sc, dI, p0, p1, **kw)


def test_detached_albedo_gradient_vs_central_differences(oracle):
    """With geometry fixed the per-seed image is a polynomial in the albedos, so FP64
    central differences pin naive AD to ~1e-7 relative."""
    sc = I.box_scene(24)
    dI = I.smooth_adjoint(sc.W, sc.H, 11)
    kw = dict(seed=3, n_paths=1 << 11, max_depth=4)
    g = oracle.gradient(sc, dI, method=oracle.NAIVE, **kw)
    a0 = sc.albedo.copy()
    for k in np.argsort(-np.abs(g["d_albedo"]))[:5]:
        h = 1e-4
        ap, am = a0.copy(), a0.copy()
        ap[k] += h
        am[k] -= h
        fd = (_loss_fd(oracle, sc, dI, (a0, sc.Le, sc.heights), (ap, sc.Le, sc.heights), **kw)
              - _loss_fd(oracle, sc, dI, (a0, sc.Le, sc.heights), (am, sc.Le, sc.heights), **kw)) / (2 * h)
        assert g["d_albedo"][k] == pytest.approx(fd, rel=1e-7, abs=1e-14)
    # emitted radiance: the image is linear in Le, so dL/dLe_c = <dI_c, I_c>/Le_c exactly
    img = oracle.render(sc, seed=3, n_paths=1 << 11, max_depth=4)
    assert np.allclose(g["d_Le"], (dI * img).sum(axis=(0, 1)) / sc.Le, rtol=1e-12)
    assert g["loss"] == pytest.approx((dI * img).sum(), rel=1e-12)


@pytest.mark.parametrize("which", ["box_hm", "slab"])
def test_attached_height_gradient_vs_frozen_central_differences(oracle, which):
    if which == "box_hm":
        sc, D = I.box_scene(24, heightmap=6), 5
    else:
        sc, D = I.slab_scene(48, n=12), 8
    dI = I.smooth_adjoint(sc.W, sc.H, 13)
    kw = dict(seed=1, n_paths=1 << 11, max_depth=D)
    g = oracle.gradient(sc, dI, method=oracle.NAIVE, attached=1, **kw)
    h0 = sc.heights.copy()
    for k in np.argsort(-np.abs(g["d_heights"]))[:4]:
        h = 1e-6
        hp, hm = h0.copy(), h0.copy()
        hp[k] += h
        hm[k] -= h
        fd = (_loss_fd(oracle, sc, dI, (sc.albedo, sc.Le, h0), (sc.albedo, sc.Le, hp), **kw)
              - _loss_fd(oracle, sc, dI, (sc.albedo, sc.Le, h0), (sc.albedo, sc.Le, hm), **kw)) / (2 * h)
        assert g["d_heights"][k] == pytest.approx(fd, rel=2e-5)
    # the attached and detached albedo gradients agree (albedo moves no vertex)
    gd = oracle.gradient(sc, dI, method=oracle.NAIVE, attached=0, **kw)
    assert np.allclose(g["d_albedo"], gd["d_albedo"], rtol=1e-12, atol=1e-300)
    assert np.allclose(g["d_Le"], gd["d_Le"], rtol=1e-12)


def test_attached_gradient_unbiased_for_derivative_of_expected_image(oracle):
    """The attached frozen-decision gradient has the expectation of d/dtheta E[<dI, I>]
    (interior derivative; no visibility boundary moves in this scene): compared with
    common-random-number central differences of the full, re-decided renderer."""
    sc = I.plane_under_light(res=16, heightmap=9, hm_std=0.05, plane_half=1.5, light_h=0.8, light_size=0.3)
    dI = np.ones((sc.H, sc.W, 3)) / (sc.W * sc.H)
    D, N, S, h = 1, 1 << 15, 32, 2e-3
    ks = [40, 31]
    h0 = sc.heights.copy()
    diffs = []
    for s in range(S):
        g = oracle.gradient(sc, dI, seed=s, n_paths=N, max_depth=D, attached=1)["d_heights"][ks]
        fd = []
        for k in ks:
            hp, hm = h0.copy(), h0.copy()
            hp[k] += h
            hm[k] -= h
            lp = oracle.gradient(sc, dI, seed=s, n_paths=N, max_depth=D, heights=hp)["loss"]
            lm = oracle.gradient(sc, dI, seed=s, n_paths=N, max_depth=D, heights=hm)["loss"]
            fd.append((lp - lm) / (2 * h))
        diffs.append(g - np.array(fd))
    d = np.array(diffs)
    z = d.mean(0) / (d.std(0, ddof=1) / np.sqrt(S))
    assert np.all(np.abs(z) < 4), z


# ------------------------------------------------------------- methods vs naive AD
def test_lrb3_restatement_equals_naive_ad_per_seed(oracle):
    """LRB-3-pass (Eq. 14-17) reaches exactly the naive reverse-mode gradient per seed."""
    sc = I.box_scene(24)
    dI = I.smooth_adjoint(sc.W, sc.H, 5)
    for seed, D in ((0, 4), (1, 9)):
        kw = dict(seed=seed, n_paths=1 << 11, max_depth=D)
        a = oracle.gradient(sc, dI, method=oracle.NAIVE, **kw)
        b = oracle.gradient(sc, dI, method=oracle.LRB3_RESTATED, **kw)
        assert np.linalg.norm(a["d_albedo"] - b["d_albedo"]) <= 1e-12 * np.linalg.norm(a["d_albedo"])
        assert np.allclose(a["d_Le"], b["d_Le"], rtol=1e-12)


def test_reslrb_restatement_equals_ad_of_reservoir_estimator(oracle):
    sc = I.box_scene(24)
    dI = I.smooth_adjoint(sc.W, sc.H, 6)
    kw = dict(seed=2, n_paths=1 << 11, max_depth=6)
    a = oracle.gradient(sc, dI, method=oracle.RESLRB_AD, **kw)
    b = oracle.gradient(sc, dI, method=oracle.RESLRB_RESTATED, **kw)
    assert np.linalg.norm(a["d_albedo"] - b["d_albedo"]) <= 1e-12 * np.linalg.norm(a["d_albedo"])
    assert np.allclose(a["d_Le"], b["d_Le"], rtol=1e-12)
    # the ResLRB primal splats the reservoir winner S = (Omega/w_R) L_R (Eq. 9); its
    # image is linear in Le too
    img = oracle.render(sc, seed=2, n_paths=1 << 11, max_depth=6, estimator=1)
    assert np.allclose(a["d_Le"], (dI * img).sum(axis=(0, 1)) / sc.Le, rtol=1e-12)


@pytest.mark.parametrize("attached", [0, 1])
def test_depth_one_all_methods_coincide(oracle, attached):
    """Depth 1: every path has at most one connection, so ResLRB selects it with weight 1
    and equals naive AD (and LRB-3) per seed."""
    sc = I.box_scene(24, heightmap=5)
    dI = I.smooth_adjoint(sc.W, sc.H, 7)
    kw = dict(seed=4, n_paths=1 << 12, max_depth=1, attached=attached)
    a = oracle.gradient(sc, dI, method=oracle.NAIVE, **kw)
    b = oracle.gradient(sc, dI, method=oracle.RESLRB_AD, **kw)
    for k in ("d_albedo", "d_Le", "d_heights"):
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-300)
    i0 = oracle.render(sc, seed=4, n_paths=1 << 12, max_depth=1)
    i1 = oracle.render(sc, seed=4, n_paths=1 << 12, max_depth=1, estimator=1)
    assert np.allclose(i0, i1, rtol=1e-12, atol=1e-300)


def test_reslrb_gradient_unbiased_paired(oracle):
    """Eq. 10: over seeds, the ResLRB gradient matches the naive gradient in expectation
    (paired per seed to cancel path noise; mean difference within 3 standard errors)."""
    sc = I.box_scene(16)
    dI = I.smooth_adjoint(sc.W, sc.H, 8)
    S = 64
    rng = np.random.default_rng(3)
    proj = rng.normal(size=sc.albedo.size)
    dd, dp = [], []
    for s in range(S):
        kw = dict(seed=1000 + s, n_paths=1 << 10, max_depth=6)
        a = oracle.gradient(sc, dI, method=oracle.NAIVE, **kw)
        b = oracle.gradient(sc, dI, method=oracle.RESLRB_AD, **kw)
        dd.append(np.concatenate([b["d_Le"] - a["d_Le"], [proj @ (b["d_albedo"] - a["d_albedo"])]]))
        dp.append(b["d_albedo"] - a["d_albedo"])
    dd = np.array(dd)
    z = dd.mean(0) / (dd.std(0, ddof=1) / np.sqrt(S))
    assert np.all(np.abs(z) < 3.5), z
    dp = np.array(dp)
    sd = dp.std(0, ddof=1)
    ok = sd > 0
    zp = dp.mean(0)[ok] / (sd[ok] / np.sqrt(S))
    assert np.mean(np.abs(zp) > 3) < 0.02
    # and it is a different per-seed estimator (variance strictly positive)
    assert np.all(dd.std(0) > 0)


# ------------------------------------------------------------------ Russian roulette
def test_russian_roulette_unbiased_and_exact(oracle):
    """Russian roulette (fixed survival probability q after a given depth) changes each
    path's estimate but not its expectation: paired per seed with the same paths without
    roulette, the image, the Le gradient and an albedo-gradient projection agree within
    3.5 standard errors; q = 1 reproduces the image bit for bit; and the roulette gradient
    stays the exact derivative of the frozen per-seed function (central differences)."""
    sc = I.box_scene(12)
    dI = I.smooth_adjoint(sc.W, sc.H, 4)
    S, kw, rr = 48, dict(n_paths=1 << 10, max_depth=8), dict(rr_depth=2, rr_prob=0.6)
    assert np.array_equal(oracle.render(sc, seed=5, **kw), oracle.render(sc, seed=5, rr_depth=2, rr_prob=1.0, **kw))
    proj = np.random.default_rng(1).normal(size=sc.albedo.size)
    diffs = []
    for s in range(S):
        g0 = oracle.gradient(sc, dI, seed=2000 + s, **kw)
        g1 = oracle.gradient(sc, dI, seed=2000 + s, **rr, **kw)
        i0 = oracle.render(sc, seed=2000 + s, **kw).sum(axis=(0, 1))
        i1 = oracle.render(sc, seed=2000 + s, **rr, **kw).sum(axis=(0, 1))
        diffs.append(np.concatenate([i1 - i0, g1["d_Le"] - g0["d_Le"], [proj @ (g1["d_albedo"] - g0["d_albedo"])]]))
    d = np.array(diffs)
    z = d.mean(0) / (d.std(0, ddof=1) / np.sqrt(S))
    assert np.all(np.abs(z) < 3.5), z
    assert np.all(d.std(0) > 0)  # the roulette changes the per-seed estimate
    g = oracle.gradient(sc, dI, seed=7, **rr, **kw)
    a0 = sc.albedo.copy()
    for k in np.argsort(-np.abs(g["d_albedo"]))[:3]:
        h = 1e-4
        ap, am = a0.copy(), a0.copy()
        ap[k] += h
        am[k] -= h
        fd = (_loss_fd(oracle, sc, dI, (a0, sc.Le, sc.heights), (ap, sc.Le, sc.heights), seed=7, **rr, **kw)
              - _loss_fd(oracle, sc, dI, (a0, sc.Le, sc.heights), (am, sc.Le, sc.heights), seed=7, **rr, **kw)) / (2 * h)
        assert g["d_albedo"][k] == pytest.approx(fd, rel=1e-7, abs=1e-14)


# ------------------------------------------------------------------ reconstruction filters
def test_gaussian_filter_definition_and_flux(oracle):
    """The wider (Gaussian) filter: nonnegative, symmetric, falling continuously to zero at
    the 1.5-pixel radius, and of unit integral, so its lattice sum averages to one over
    film positions (as the tent's is one everywhere); an image's total flux is therefore
    the tent image's up to the lattice ripple, and attached derivatives through the filter
    stay exact (central differences of the frozen function)."""
    rng = np.random.default_rng(0)
    sums = []
    for ux, uy in rng.uniform(20, 40, size=(4000, 2)):
        px, py, w = oracle.filter_taps(1, 64, 64, ux, uy)
        assert len(w) <= 9 and np.all(w >= 0)
        sums.append(w.sum())
        tpx, tpy, tw = oracle.filter_taps(0, 64, 64, ux, uy)
        assert tw.sum() == pytest.approx(1.0, abs=1e-12)
    assert np.mean(sums) == pytest.approx(1.0, abs=2e-3)
    assert np.std(sums) < 0.05
    # symmetry and continuity at the radius: a tap entering at distance 1.5 has weight ~0
    _, _, wa = oracle.filter_taps(1, 64, 64, 30.5 + 0.3, 30.5)
    _, _, wb = oracle.filter_taps(1, 64, 64, 30.5 - 0.3, 30.5)
    assert np.allclose(np.sort(wa), np.sort(wb), atol=1e-15)
    _, _, we = oracle.filter_taps(1, 64, 64, 30.5 + 1.5 - 1e-9, 30.5)
    assert we.min() < 1e-7
    sc = I.box_scene(20)
    kw = dict(seed=3, n_paths=1 << 14, max_depth=4)
    flux_t = oracle.render(sc, **kw).sum()
    flux_g = oracle.render(sc, filter=1, **kw).sum()
    # the wider filter loses a little more at the film border (taps off the film drop)
    assert flux_g == pytest.approx(flux_t, rel=1e-2) and flux_g <= flux_t
    hsc = I.box_scene(16, heightmap=4, hm_std=0.04)
    dI = I.smooth_adjoint(hsc.W, hsc.H, 12)
    kw = dict(seed=4, n_paths=1 << 9, max_depth=4, filter=1)
    g = oracle.gradient(hsc, dI, attached=1, **kw)
    h0 = hsc.heights.copy()
    for k in np.argsort(-np.abs(g["d_heights"]))[:3]:
        e = 1e-5
        hp, hm = h0.copy(), h0.copy()
        hp[k] += e
        hm[k] -= e
        p0 = (hsc.albedo, hsc.Le, h0)
        fd = (_loss_fd(oracle, hsc, dI, p0, (hsc.albedo, hsc.Le, hp), **kw)
              - _loss_fd(oracle, hsc, dI, p0, (hsc.albedo, hsc.Le, hm), **kw)) / (2 * e)
        assert g["d_heights"][k] == pytest.approx(fd, rel=2e-5, abs=1e-12)


# ------------------------------------------------------------------ learned target MLP
def _mlp_params(seed=0):
    rng = np.random.default_rng(seed)
    P = np.zeros(5352)
    P[0:1024] = rng.normal(size=1024) * np.sqrt(2 / 16)
    P[1024:1088] = rng.normal(size=64) * 0.1
    P[1088:5184] = rng.normal(size=4096) * np.sqrt(2 / 64)
    P[5184:5248] = rng.normal(size=64) * 0.1
    P[5248:5312] = rng.normal(size=64) * np.sqrt(1 / 64)
    P[5312] = 0.3
    P[5313:5329] = rng.normal(size=16) * 0.1
    P[5329:5345] = rng.uniform(0.5, 2.0, size=16)
    P[5345], P[5346] = 1.7, -0.4
    return P


def test_mlp_oracle_gradient_vs_central_differences(oracle):
    """The oracle network's reverse mode (FP64, no rounding) against central differences of
    its loss, on every parameter group."""
    rng = np.random.default_rng(1)
    P = _mlp_params(0)
    X = rng.normal(size=(40, 16))
    T = rng.normal(size=40)
    g, loss = oracle.mlp_grad(P, X, T, round_bf16=False)
    for k in [3, 500, 1030, 1088 + 7 * 64 + 9, 4000, 5190, 5250, 5312]:
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (oracle.mlp_grad(Pp, X, T, round_bf16=False)[1] - oracle.mlp_grad(Pm, X, T, round_bf16=False)[1]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # the forward is the plain network: one sample by hand
    x = ((X[0].astype(np.float32) - P[5313:5329].astype(np.float32)) * P[5329:5345].astype(np.float32)).astype(np.float64)
    h1 = np.maximum(P[1024:1088] + x @ P[0:1024].reshape(16, 64), 0)
    h2 = np.maximum(P[5184:5248] + h1 @ P[1088:5184].reshape(64, 64), 0)
    y = P[5312] + h2 @ P[5248:5312]
    assert oracle.mlp_forward(P, X[:1], round_bf16=False)[0] == pytest.approx(y, rel=1e-12)


def test_mlp_oracle_bf16_rounding():
    """BFloat16 emulation: each rounding keeps 8 significant bits (relative error <= 2^-9),
    so over 64-term sums the network output moves by well under a few percent of its
    typical magnitude, and it does move."""
    from oracle import oracle as O
    P = _mlp_params(2)
    X = np.random.default_rng(3).normal(size=(64, 16))
    a = O.mlp_forward(P, X, round_bf16=True)
    b = O.mlp_forward(P, X, round_bf16=False)
    rel = np.abs(a - b) / np.abs(b).mean()
    assert np.median(rel) < 1e-2 and np.max(rel) < 5e-2
    assert not np.allclose(a, b, rtol=1e-6)


def test_filter_kink_distance_query(oracle):
    """The per-path distance to the nearest pixel centre (where the tent filter's derivative
    jumps) equals, for a path with exactly one connection, the distance of that connection's
    film coordinates read from the reservoir records (which then hold the only candidate);
    paths without a connection report 1e9, and the image equals the plain estimator's."""
    sc = I.box_scene(24)
    kw = dict(seed=5, n_paths=1 << 11, max_depth=3)
    img3, kr = oracle.render(sc, estimator=3, want_records=True, **kw)
    img0 = oracle.render(sc, **kw)
    assert np.array_equal(img3, img0)
    _, rr = oracle.render(sc, estimator=1, want_records=True, **kw)
    n_conn = rr[:, 7]
    one = (n_conn == 1) & (rr[:, 0] >= 0)
    assert one.sum() > 100
    u = rr[one, 2:4]
    d = np.abs((u - 0.5) - np.round(u - 0.5)).min(axis=1)
    assert np.allclose(kr[one, 0], d, rtol=0, atol=1e-12)
    assert np.all(kr[n_conn == 0, 0] == 1e9)
    assert np.all((kr[n_conn > 0, 0] >= 0) & (kr[n_conn > 0, 0] <= 0.5))


def test_connection_query_reproduces_image_and_adjoints(oracle):
    """The per-connection query (the source of the learned target's reference pairs) holds the
    same connections the image and the gradient use: splatting its L at its u gives the
    rendered image, its Lbar . L summed per path gives each path's delta_total (Eq. 14), its
    counts the connection counts; and each row is geometrically consistent (unit normal and
    direction, the normal on the arrival side, L = throughput x albedo x connection weight
    for the uniform albedo of the height field)."""
    sc = I.box_scene(24, heightmap=5, hm_std=0.03)
    dI = I.smooth_adjoint(sc.W, sc.H, 9)
    kw = dict(seed=6, n_paths=1 << 11, max_depth=5)
    rows = oracle.connections(sc, dI, **kw)
    img = oracle.render(sc, **kw)
    acc = np.zeros_like(img)
    for r in rows:
        px, py, w = oracle.filter_taps(0, sc.W, sc.H, r[14], r[15])
        for x, y, ww in zip(px, py, w):
            acc[y, x] += ww * r[17:20]
    assert np.allclose(acc, img, rtol=1e-12, atol=1e-15)
    g = oracle.gradient(sc, dI, want_dbg=True, **kw)
    per_path = np.zeros((kw["n_paths"], 3))
    np.add.at(per_path, rows[:, 0].astype(int), rows[:, 20:23] * rows[:, 17:20])
    assert np.allclose(per_path, g["dbg"][:, :3], rtol=1e-12, atol=1e-18)
    assert np.array_equal(np.bincount(rows[:, 0].astype(int), minlength=kw["n_paths"]), g["dbg"][:, 3])
    assert np.allclose(np.linalg.norm(rows[:, 5:8], axis=1), 1, atol=1e-12)
    assert np.allclose(np.linalg.norm(rows[:, 8:11], axis=1), 1, atol=1e-12)
    assert np.all(np.einsum("ij,ij->i", rows[:, 5:8], rows[:, 8:11]) < 0)
    x, y, z = rows[:, 2], rows[:, 3], rows[:, 4]
    hm = (x > 0.26) & (x < 0.74) & (z > 0.26) & (z < 0.74) & (y > 0.1) & (y < 0.4)  # the height field (albedo 0.5)
    assert hm.sum() > 10
    assert np.allclose(rows[hm, 17:20], rows[hm, 11:14] * 0.5 * rows[hm, 16:17], rtol=1e-12)


def test_bidirectional_estimator_unbiased_and_exact(oracle):
    """The bidirectional estimator (light-tracer connections and camera samples with
    next-event estimation, balance heuristic): without camera samples it is the light
    tracer exactly; its expectation is the light tracer's, and so is that of the camera
    samples alone (per-pixel z-scores over 16 seeds; a wrong density ratio would leave the
    two strategies' weights not summing to one and bias the image); its naive-AD gradient
    equals central differences of its own image (detached: a polynomial in the albedos with
    weights that depend on geometry only) and is linear in Le."""
    sc = I.box_scene(16)
    D = 3
    dI = I.smooth_adjoint(sc.W, sc.H, 17)
    assert np.array_equal(oracle.render_bidir(sc, 0, seed=1, n_paths=1 << 12, max_depth=D),
                          oracle.render(sc, seed=1, n_paths=1 << 12, max_depth=D))
    g0 = oracle.gradient_bidir(sc, dI, 0, seed=1, n_paths=1 << 12, max_depth=D)
    g1 = oracle.gradient(sc, dI, seed=1, n_paths=1 << 12, max_depth=D)
    assert np.allclose(g0["d_albedo"], g1["d_albedo"], rtol=1e-12, atol=1e-300)
    assert np.allclose(g0["d_Le"], g1["d_Le"], rtol=1e-12)
    S = 16
    lt = np.array([oracle.render(sc, seed=100 + s, n_paths=1 << 14, max_depth=D) for s in range(S)])
    for n_light, base in ((1 << 14, 200), (0, 300)):
        bi = np.array([oracle.render_bidir(sc, 1 << 14, seed=base + s, n_paths=n_light, max_depth=D)
                       for s in range(S)])
        d = bi.mean(0) - lt.mean(0)
        se = np.sqrt(lt.var(0, ddof=1) / S + bi.var(0, ddof=1) / S)
        z = d[se > 0] / se[se > 0]
        assert 0.8 < np.mean(z * z) < 1.35 and np.abs(z).max() < 4.5, (n_light, np.mean(z * z), np.abs(z).max())
    kw = dict(seed=5, n_paths=1 << 11, max_depth=D)
    g = oracle.gradient_bidir(sc, dI, 1 << 11, **kw)
    rng = np.random.default_rng(2)
    v = rng.normal(size=sc.albedo.size)
    h = 1e-3

    def loss(a):
        return (oracle.render_bidir(sc, 1 << 11, albedo=a, **kw) * dI).sum()
    fd = (loss(sc.albedo + h * v) - loss(sc.albedo - h * v)) / (2 * h)
    assert g["d_albedo"] @ v == pytest.approx(fd, rel=1e-7)
    img = oracle.render_bidir(sc, 1 << 11, **kw)
    assert np.allclose(g["d_Le"], (dI * img).sum(axis=(0, 1)) / sc.Le, rtol=1e-12)
    assert g["loss"] == pytest.approx((dI * img).sum(), rel=1e-12)


def test_literal_attached_variant_exact_on_first_chains_and_unbiased_with_noise(oracle):
    """The paper-literal attached LRB-3 (film-position transport by accumulated two-point
    Jacobians with the determinant-guarded inverse, Eq. 18-19 and Sec. 5): on the caustic slab
    at depth 3 every specular chain starts at the emitter (the accumulated Jacobian stays
    invertible), where it equals naive AD of the exact model per seed; a path whose chain
    starts after a diffuse vertex (singular accumulated Jacobian) loses its transport with
    the guard alone (here most of its height gradient) and recovers it in expectation with
    the zero-mean Jacobian noise (per-parameter z over 256 noise draws; the relative
    determinant guard set low, so that it leaves every noisy product to the inverse)."""
    sc = I.slab_scene(48, n=12)
    dI = I.smooth_adjoint(sc.W, sc.H, 61)
    kw = dict(seed=11, n_paths=1 << 12, max_depth=3)
    a = oracle.gradient(sc, dI, attached=1, **kw)
    b = oracle.gradient_literal(sc, dI, **kw)
    for k in ("d_heights", "d_Le", "d_albedo"):
        assert np.linalg.norm(b[k] - a[k]) <= 1e-12 * np.linalg.norm(a[k]), k
    for p in (2064, 3619):  # paths of this scene and seed with such a chain ending in a connection
        kw = dict(seed=11, n_paths=1, path_begin=p, n_norm=1 << 12, max_depth=8, n_threads=1)
        ref = oracle.gradient(sc, dI, attached=1, **kw)["d_heights"]
        guard = oracle.gradient_literal(sc, dI, **kw)["d_heights"]
        assert np.linalg.norm(guard - ref) > 0.5 * np.linalg.norm(ref)
        G = np.array([oracle.gradient_literal(sc, dI, jac_noise=True, noise_seed=s, det_eps=1e-10, **kw)["d_heights"]
                      for s in range(256)])
        d = G - ref
        sd = d.std(0, ddof=1)
        ok = sd > 1e-9 * np.abs(ref).max()
        z = d.mean(0)[ok] / (sd[ok] / np.sqrt(len(G)))
        assert ok.sum() >= 3 and np.abs(z).max() < 4.0, np.abs(z).max()
        assert np.abs(d.mean(0)[~ok]).max(initial=0.0) < 1e-12 * np.abs(ref).max()
