"""ctypes wrapper of the FP64 CPU oracle (``lt_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this module; the product path never does.  It
shares no code with the CUDA implementation; only the seeded scene generators
(``paper_2609_32920_gb300.inputs``) feed both.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lt_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

NAIVE, LRB3_RESTATED, RESLRB_AD, RESLRB_RESTATED = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with the host compiler (plain g++, no GPU code)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-Wno-dangling-pointer", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


class or_scene(C.Structure):
    _fields_ = [("n_quads", C.c_int), ("quads", C.POINTER(C.c_double)),
                ("n_verts", C.c_int), ("verts", C.POINTER(C.c_double)), ("vert_h", C.POINTER(C.c_int)),
                ("n_tris", C.c_int), ("tris", C.POINTER(C.c_int)), ("prim_mat", C.POINTER(C.c_int)),
                ("n_mats", C.c_int), ("mat_type", C.POINTER(C.c_int)), ("mat_ior", C.POINTER(C.c_double)),
                ("mat_tex_off", C.POINTER(C.c_int)), ("mat_tex_w", C.POINTER(C.c_int)),
                ("mat_tex_h", C.POINTER(C.c_int)), ("emitter_quad", C.c_int),
                ("cam_pos", C.c_double * 3), ("cam_look", C.c_double * 3), ("cam_up", C.c_double * 3),
                ("fov_y_deg", C.c_double), ("W", C.c_int), ("H", C.c_int)]


class or_params(C.Structure):
    _fields_ = [("albedo", C.POINTER(C.c_double)), ("n_albedo", C.c_int), ("Le", C.POINTER(C.c_double)),
                ("heights", C.POINTER(C.c_double)), ("n_heights", C.c_int)]


class or_run(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("path_begin", C.c_int64), ("n_paths", C.c_int64),
                ("n_norm", C.c_int64), ("max_depth", C.c_int), ("method", C.c_int),
                ("attached", C.c_int), ("n_threads", C.c_int), ("rr_depth", C.c_int), ("rr_q", C.c_double),
                ("filter", C.c_int)]


class or_grads(C.Structure):
    _fields_ = [("d_albedo", C.POINTER(C.c_double)), ("d_Le", C.POINTER(C.c_double)),
                ("d_heights", C.POINTER(C.c_double)), ("loss", C.POINTER(C.c_double))]


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = LIB if os.path.exists(LIB) else build()
            L = C.CDLL(path)
            P = C.POINTER
            L.or_render_lt.argtypes = [P(or_scene), P(or_params), P(or_run), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int, C.c_void_p]
            L.or_gradient.argtypes = [P(or_scene), P(or_params), P(or_run), C.c_void_p, C.c_void_p,
                                      P(or_grads), C.c_void_p, C.c_void_p]
            L.or_frozen_loss.argtypes = [P(or_scene), P(or_params), P(or_params), P(or_run), C.c_void_p,
                                         C.c_void_p]
            L.or_frozen_loss.restype = C.c_double
            L.or_render_pt.argtypes = [P(or_scene), P(or_params), C.c_uint64, C.c_int, C.c_int, C.c_int,
                                       C.c_void_p]
            L.or_philox.argtypes = [C.c_uint32, C.c_uint32, C.c_void_p, C.c_void_p]
            L.or_filter_taps.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_void_p,
                                         C.c_void_p, C.c_void_p]
            L.or_uniforms.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_void_p]
            L.or_dielectric.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
            L.or_reservoir.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            L.or_reservoir.restype = C.c_int
            L.or_intersect.argtypes = [P(or_scene), P(or_params), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
            L.or_intersect.restype = C.c_int
            L.or_render_bidir.argtypes = [P(or_scene), P(or_params), P(or_run), C.c_int64, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_gradient_bidir.argtypes = [P(or_scene), P(or_params), P(or_run), C.c_int64, C.c_void_p,
                                            C.c_void_p, C.c_void_p, P(or_grads)]
            L.or_gradient_literal.argtypes = [P(or_scene), P(or_params), P(or_run), C.c_void_p, C.c_void_p,
                                              C.c_int, C.c_uint64, C.c_double, C.c_double, P(or_grads)]
            L.or_connections.argtypes = [P(or_scene), P(or_params), P(or_run), C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_int64]
            L.or_connections.restype = C.c_int64
            L.or_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p]
            L.or_mlp_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p]
            L.or_mlp_grad.restype = C.c_double
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class _Bound:
    """Keeps the numpy arrays alive while ctypes structs point at them."""

    def __init__(self, scene, albedo=None, Le=None, heights=None):
        s = scene
        self.keep = []

        def f64(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self.keep.append(a)
            return a

        def i32(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            self.keep.append(a)
            return a

        q, v, vh, t, pm = f64(s.quads.reshape(-1)), f64(s.verts.reshape(-1)), i32(s.vert_h), i32(s.tris.reshape(-1)), i32(s.prim_mat)
        mt, mi, mo, mw, mh = i32(s.mat_type), f64(s.mat_ior), i32(s.mat_tex_off), i32(s.mat_tex_w), i32(s.mat_tex_h)
        self.sc = or_scene(s.n_quads, _dp(q), s.verts.shape[0], _dp(v), _ip(vh), s.n_tris, _ip(t), _ip(pm),
                           len(s.mat_type), _ip(mt), _dp(mi), _ip(mo), _ip(mw), _ip(mh), s.emitter_quad,
                           (C.c_double * 3)(*s.cam_pos), (C.c_double * 3)(*s.cam_look), (C.c_double * 3)(*s.cam_up),
                           s.fov_y_deg, s.W, s.H)
        self.params = self.make_params(s.albedo if albedo is None else albedo, s.Le if Le is None else Le,
                                       s.heights if heights is None else heights)

    def make_params(self, albedo, Le, heights):
        a = np.ascontiguousarray(albedo, dtype=np.float64)
        le = np.ascontiguousarray(Le, dtype=np.float64)
        h = np.ascontiguousarray(heights, dtype=np.float64)
        if h.size == 0:
            h = np.zeros(1)
        self.keep += [a, le, h]
        return or_params(_dp(a), a.size, _dp(le), _dp(h), int(np.asarray(heights).size))


def _threads(n):
    return int(n) if n else max(1, min(os.cpu_count() or 1, 64))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _rr(rr_depth, rr_prob):
    """Russian roulette settings; the survival probability is rounded to FP32 as the CUDA
    path stores it, so both take the same survival decisions."""
    return int(rr_depth), float(np.float32(rr_prob))


def render(scene, seed=0, n_paths=1 << 12, max_depth=4, path_begin=0, n_norm=0, estimator=0, mask=None,
           want_hash=False, want_records=False, n_threads=0, albedo=None, Le=None, heights=None, rr_depth=0,
           rr_prob=1.0, filter=0):
    """Light-traced image [H, W, 3] (float64).  estimator 0 = every connection, 1 = reservoir."""
    b = _Bound(scene, albedo, Le, heights)
    img = np.zeros((scene.H, scene.W, 3))
    run = or_run(seed, path_begin, n_paths, n_norm or n_paths, max_depth, 0, 0, _threads(n_threads),
                 *_rr(rr_depth, rr_prob), int(filter))
    hashes = np.zeros(n_paths, dtype=np.uint32) if want_hash else None
    recs = np.zeros((n_paths, 8)) if want_records else None
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    lib().or_render_lt(C.byref(b.sc), C.byref(b.params), C.byref(run), _ptr(m), img.ctypes.data,
                       _ptr(hashes), estimator, _ptr(recs))
    out = [img]
    if want_hash:
        out.append(hashes)
    if want_records:
        out.append(recs)
    return out[0] if len(out) == 1 else tuple(out)


def gradient(scene, dI, seed=0, n_paths=1 << 12, max_depth=4, method=NAIVE, attached=0, path_begin=0, n_norm=0,
             mask=None, want_hash=False, want_dbg=False, n_threads=0, albedo=None, Le=None, heights=None,
             rr_depth=0, rr_prob=1.0, filter=0):
    """dict(d_albedo, d_Le, d_heights, loss[, hash][, dbg]) of <dI, I_s>."""
    b = _Bound(scene, albedo, Le, heights)
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    assert dI.shape == (scene.H, scene.W, 3)
    ga = np.zeros(max(1, scene.albedo.size))
    gl = np.zeros(3)
    gh = np.zeros(max(1, scene.heights.size))
    loss = np.zeros(1)
    g = or_grads(_dp(ga), _dp(gl), _dp(gh), _dp(loss))
    run = or_run(seed, path_begin, n_paths, n_norm or n_paths, max_depth, method, attached, _threads(n_threads),
                 *_rr(rr_depth, rr_prob), int(filter))
    hashes = np.zeros(n_paths, dtype=np.uint32) if want_hash else None
    dbg = np.zeros((n_paths, 4)) if want_dbg else None
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    rc = lib().or_gradient(C.byref(b.sc), C.byref(b.params), C.byref(run), dI.ctypes.data, _ptr(m), C.byref(g),
                           _ptr(hashes), _ptr(dbg))
    if rc != 0:
        raise ValueError(f"oracle or_gradient refused (code {rc})")
    out = dict(d_albedo=ga[:scene.albedo.size], d_Le=gl, d_heights=gh[:scene.heights.size], loss=float(loss[0]))
    if want_hash:
        out["hash"] = hashes
    if want_dbg:
        out["dbg"] = dbg
    return out


def connections(scene, dI, seed=0, n_paths=1 << 12, max_depth=4, path_begin=0, n_norm=0, mask=None, cap=1 << 20,
                filter=0):
    """Every valid sensor connection [n, 24]: path, vertex index k, x[3], arrival-side normal[3],
    arrival direction[3], throughput before the albedo[3], u_x, u_y, connection weight,
    L[3], Lbar[3], 0 (see or_connections)."""
    b = _Bound(scene)
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    run = or_run(seed, path_begin, n_paths, n_norm or n_paths, max_depth, 0, 0, 1, 0, 1.0, int(filter))
    rows = np.zeros((cap, 24))
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    k = lib().or_connections(C.byref(b.sc), C.byref(b.params), C.byref(run), dI.ctypes.data, _ptr(m),
                             rows.ctypes.data, cap)
    return rows[: min(k, cap)]


def gradient_literal(scene, dI, seed=0, n_paths=1 << 12, max_depth=4, path_begin=0, n_norm=0, mask=None,
                     jac_noise=False, noise_seed=0, sigma=1.0, det_eps=1e-6, n_threads=0, filter=0):
    """dict(d_albedo, d_Le, d_heights, loss): the paper-literal attached LRB-3 gradient
    (film-position transport by accumulated two-point Jacobians with the determinant-guarded
    inverse, optional Jacobian noise; see or_gradient_literal)."""
    b = _Bound(scene)
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    ga = np.zeros(max(1, scene.albedo.size))
    gl = np.zeros(3)
    gh = np.zeros(max(1, scene.heights.size))
    loss = np.zeros(1)
    g = or_grads(_dp(ga), _dp(gl), _dp(gh), _dp(loss))
    run = or_run(seed, path_begin, n_paths, n_norm or n_paths, max_depth, 0, 1, _threads(n_threads), 0, 1.0,
                 int(filter))
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    rc = lib().or_gradient_literal(C.byref(b.sc), C.byref(b.params), C.byref(run), dI.ctypes.data, _ptr(m),
                                   int(bool(jac_noise)), int(noise_seed), float(sigma), float(det_eps), C.byref(g))
    if rc != 0:
        raise ValueError(f"oracle or_gradient_literal refused (code {rc})")
    return dict(d_albedo=ga[:scene.albedo.size], d_Le=gl, d_heights=gh[:scene.heights.size], loss=float(loss[0]))


def render_bidir(scene, n_cam, seed=0, n_paths=1 << 12, max_depth=4, n_norm=0, mask=None, cam_mask=None,
                 want_hash=False, n_threads=0, filter=0, albedo=None, Le=None):
    """Bidirectional image [H, W, 3]: light-tracer connections of n_paths light paths and
    n_cam camera samples with next-event estimation, balance heuristic (detached, diffuse
    scenes).  want_hash: also (light path hashes, camera sample hashes)."""
    b = _Bound(scene, albedo, Le)
    img = np.zeros((scene.H, scene.W, 3))
    run = or_run(seed, 0, n_paths, n_norm or n_paths, max_depth, 0, 0, _threads(n_threads), 0, 1.0, int(filter))
    lh = np.zeros(max(1, n_paths), dtype=np.uint32)
    ch = np.zeros(max(1, n_cam), dtype=np.uint32)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    cm = None if cam_mask is None else np.ascontiguousarray(cam_mask, dtype=np.uint8)
    rc = lib().or_render_bidir(C.byref(b.sc), C.byref(b.params), C.byref(run), int(n_cam), _ptr(m), _ptr(cm),
                               img.ctypes.data, lh.ctypes.data, ch.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle or_render_bidir refused (code {rc})")
    return (img, lh[:n_paths], ch[:n_cam]) if want_hash else img


def gradient_bidir(scene, dI, n_cam, seed=0, n_paths=1 << 12, max_depth=4, n_norm=0, mask=None, cam_mask=None,
                   n_threads=0, filter=0, albedo=None, Le=None):
    """dict(d_albedo, d_Le, loss) of <dI, I_bidir>: naive tape AD of the bidirectional
    estimator of render_bidir."""
    b = _Bound(scene, albedo, Le)
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    ga = np.zeros(max(1, scene.albedo.size))
    gl = np.zeros(3)
    gh = np.zeros(max(1, scene.heights.size))
    loss = np.zeros(1)
    g = or_grads(_dp(ga), _dp(gl), _dp(gh), _dp(loss))
    run = or_run(seed, 0, n_paths, n_norm or n_paths, max_depth, 0, 0, _threads(n_threads), 0, 1.0, int(filter))
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    cm = None if cam_mask is None else np.ascontiguousarray(cam_mask, dtype=np.uint8)
    rc = lib().or_gradient_bidir(C.byref(b.sc), C.byref(b.params), C.byref(run), int(n_cam), dI.ctypes.data,
                                 _ptr(m), _ptr(cm), C.byref(g))
    if rc != 0:
        raise ValueError(f"oracle or_gradient_bidir refused (code {rc})")
    return dict(d_albedo=ga[:scene.albedo.size], d_Le=gl, loss=float(loss[0]))


def frozen_loss(scene, dI, params0, params1, seed=0, n_paths=1 << 10, max_depth=4, method=NAIVE, path_begin=0,
                n_norm=0, mask=None, n_threads=0, rr_depth=0, rr_prob=1.0, filter=0):
    """<dI, I_s> with decisions frozen at params0=(albedo, Le, heights) and values at params1."""
    b = _Bound(scene)
    p0 = b.make_params(*params0)
    p1 = b.make_params(*params1)
    dI = np.ascontiguousarray(dI, dtype=np.float64)
    run = or_run(seed, path_begin, n_paths, n_norm or n_paths, max_depth, method, 0, _threads(n_threads),
                 *_rr(rr_depth, rr_prob), int(filter))
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    return float(lib().or_frozen_loss(C.byref(b.sc), C.byref(p0), C.byref(p1), C.byref(run), dI.ctypes.data,
                                      _ptr(m)))


def render_pt(scene, seed=0, spp=64, max_depth=4, n_threads=0):
    b = _Bound(scene)
    img = np.zeros((scene.H, scene.W, 3))
    lib().or_render_pt(C.byref(b.sc), C.byref(b.params), seed, spp, max_depth, _threads(n_threads), img.ctypes.data)
    return img


def philox(key, ctr):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox(int(key[0]), int(key[1]), c.ctypes.data, o.ctypes.data)
    return o


def filter_taps(filter, W, H, ux, uy):
    """(px, py, w) of the reconstruction filter's taps at film position (ux, uy)."""
    px, py, w = np.zeros(9, dtype=np.int32), np.zeros(9, dtype=np.int32), np.zeros(9)
    k = lib().or_filter_taps(int(filter), int(W), int(H), float(ux), float(uy), px.ctypes.data, py.ctypes.data,
                             w.ctypes.data)
    return px[:k], py[:k], w[:k]


def uniforms(seed, n, d, s=0):
    o = np.zeros(4)
    lib().or_uniforms(seed, n, d, s, o.ctypes.data)
    return o


def dielectric(din, n, ior, u):
    d = np.ascontiguousarray(din, dtype=np.float64)
    nn = np.ascontiguousarray(n, dtype=np.float64)
    out = np.zeros(3)
    F = np.zeros(1)
    r = np.zeros(1, dtype=np.int32)
    lib().or_dielectric(d.ctypes.data, nn.ctypes.data, ior, u, out.ctypes.data, F.ctypes.data, r.ctypes.data)
    return out, float(F[0]), bool(r[0])


def reservoir(weights, us):
    w = np.ascontiguousarray(weights, dtype=np.float64)
    u = np.ascontiguousarray(us, dtype=np.float64)
    rw = np.zeros(1)
    R = lib().or_reservoir(w.ctypes.data, w.size, u.ctypes.data, rw.ctypes.data)
    return R, float(rw[0])


def intersect(scene, org, dir, skip=-1):
    b = _Bound(scene)
    o = np.ascontiguousarray(org, dtype=np.float64)
    d = np.ascontiguousarray(dir, dtype=np.float64)
    out = np.zeros(3)
    prim = lib().or_intersect(C.byref(b.sc), C.byref(b.params), o.ctypes.data, d.ctypes.data, skip, out.ctypes.data)
    return prim, out


def mlp_forward(P, X, round_bf16=True):
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 16)
    out = np.zeros(X.shape[0])
    lib().or_mlp_forward(P.ctypes.data, X.ctypes.data, X.shape[0], int(round_bf16), out.ctypes.data)
    return out


def mlp_grad(P, X, T, round_bf16=True):
    P = np.ascontiguousarray(P, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 16)
    T = np.ascontiguousarray(T, dtype=np.float64)
    g = np.zeros(5313)
    loss = lib().or_mlp_grad(P.ctypes.data, X.ctypes.data, T.ctypes.data, X.shape[0], int(round_bf16), g.ctypes.data)
    return g, float(loss)
