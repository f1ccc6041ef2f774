"""Thin Python binding of liblt (include/lt.h): argument marshalling only.

Every step of the light-tracing path runs in the library's CUDA kernels; PyTorch only
supplies device memory and the current CUDA stream.  There is no CPU fallback: if the
compiled library is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import inputs as _inputs

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblt.so")

LT_OK, LT_ERR_INVALID_ARG, LT_ERR_OOM, LT_ERR_CUDA, LT_ERR_TIMEOUT, LT_ERR_DEVICE_CHECK, LT_ERR_UNSUPPORTED = range(7)
EST_PLAIN, EST_RESLRB, EST_NAIVE, EST_BUFFERED = 0, 1, 2, 3
TARGET_LUMINANCE, TARGET_MLP = 0, 1
STATUS_NAMES = {0: "LT_OK", 1: "LT_ERR_INVALID_ARG", 2: "LT_ERR_OOM", 3: "LT_ERR_CUDA", 4: "LT_ERR_TIMEOUT",
                5: "LT_ERR_DEVICE_CHECK", 6: "LT_ERR_UNSUPPORTED"}


class LTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


F3 = C.c_float * 3


class lt_scene_desc(C.Structure):
    _fields_ = [("n_quads", C.c_int), ("quads", C.c_void_p), ("n_verts", C.c_int), ("verts", C.c_void_p),
                ("vert_h", C.c_void_p), ("n_tris", C.c_int), ("tris", C.c_void_p), ("prim_mat", C.c_void_p),
                ("n_mats", C.c_int), ("mat_type", C.c_void_p), ("mat_ior", C.c_void_p),
                ("mat_tex_off", C.c_void_p), ("mat_tex_w", C.c_void_p), ("mat_tex_h", C.c_void_p),
                ("emitter_quad", C.c_int), ("cam_pos", F3), ("cam_look", F3), ("cam_up", F3),
                ("fov_y_deg", C.c_float), ("width", C.c_int), ("height", C.c_int), ("n_albedo", C.c_int),
                ("n_heights", C.c_int)]


class lt_params(C.Structure):
    _fields_ = [("albedo", C.c_void_p), ("Le", C.c_void_p)]


class lt_render_opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("path_offset", C.c_int64), ("n_paths", C.c_int64), ("n_norm", C.c_int64),
                ("max_depth", C.c_int), ("attached", C.c_int), ("target", C.c_int), ("mlp", C.c_void_p),
                ("block_size", C.c_int), ("blocks_per_sm", C.c_int), ("path_mask", C.c_void_p),
                ("path_hash", C.c_void_p), ("path_dbg", C.c_void_p), ("census", C.c_void_p),
                ("lrb3_state", C.c_void_p), ("lrb3_state_bytes", C.c_size_t), ("lrb3_mask_ready", C.c_int),
                ("rr_depth", C.c_int), ("rr_prob", C.c_float), ("filter", C.c_int), ("bvh_width", C.c_int),
                ("scatter", C.c_int), ("literal", C.c_int), ("jac_noise", C.c_int), ("noise_seed", C.c_uint64),
                ("det_eps", C.c_float)]


class lt_grads(C.Structure):
    _fields_ = [("d_albedo", C.c_void_p), ("d_Le", C.c_void_p), ("d_heights", C.c_void_p), ("accumulate", C.c_int)]


class lt_batch_item(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("params", lt_params), ("heights", C.c_void_p), ("opts", lt_render_opts),
                ("image", C.c_void_p), ("records", C.c_void_p), ("d_image", C.c_void_p), ("grads", lt_grads)]


class lt_bidir_opts(C.Structure):
    _fields_ = [("n_cam", C.c_int64), ("cam_mask", C.c_void_p), ("cam_hash", C.c_void_p)]


class lt_batch_config(C.Structure):
    _fields_ = [("block_size", C.c_int), ("paths_per_thread", C.c_int), ("blocks_per_sm", C.c_int),
                ("bvh_width", C.c_int)]


PASS_PRIMAL, PASS_PRIMAL_RESLRB, PASS_LRB3, PASS_RESLRB = 0, 1, 2, 3

_lib = None
_lock = threading.Lock()

# Every symbol include/lt.h declares (checked by the CPU test-suite against the .so).
EXPORTS = ["lt_scene_create", "lt_scene_refit", "lt_scene_destroy", "lt_primal", "lt_backward_lrb3",
           "lt_backward_reslrb", "lt_backward_naive", "lt_film_l2", "lt_record_size", "lt_naive_workspace_bytes",
           "lt_sync_status", "lt_last_error", "lt_version", "lt_mlp_collect", "lt_mlp_init_stats", "lt_mlp_grad",
           "lt_mlp_adam", "lt_mlp_forward", "lt_naive_gradient_static", "lt_batch_create", "lt_batch_run",
           "lt_batch_set_config", "lt_batch_get_config", "lt_batch_tune", "lt_batch_destroy", "lt_lrb3_state_bytes",
           "lt_backward_lrb2", "lt_lrb2_buffer_bytes", "lt_bidir_primal", "lt_bidir_backward"]
MLP_PARAMS, MLP_WEIGHTS = 5352, 5313


def lib():
    """Load liblt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise LTError(LT_ERR_UNSUPPORTED, f"{LIB_PATH} is missing: build it with paper_2609_32920_gb300.build")
            L = C.CDLL(LIB_PATH)
            P, V = C.POINTER, C.c_void_p
            L.lt_scene_create.argtypes = [P(lt_scene_desc), V, P(V)]
            L.lt_scene_refit.argtypes = [V, V, V]
            L.lt_scene_destroy.argtypes = [V]
            L.lt_scene_destroy.restype = None
            L.lt_primal.argtypes = [V, P(lt_params), P(lt_render_opts), C.c_int, V, V, C.c_size_t, V]
            L.lt_backward_lrb3.argtypes = [V, P(lt_params), P(lt_render_opts), V, P(lt_grads), V]
            L.lt_backward_reslrb.argtypes = [V, P(lt_params), P(lt_render_opts), V, V, P(lt_grads), V]
            L.lt_backward_naive.argtypes = [V, P(lt_params), P(lt_render_opts), V, V, C.c_size_t, P(lt_grads), V]
            L.lt_film_l2.argtypes = [V, V, C.c_int64, V, V, V]
            L.lt_record_size.argtypes = [P(lt_render_opts)]
            L.lt_record_size.restype = C.c_size_t
            L.lt_naive_workspace_bytes.argtypes = [P(lt_render_opts)]
            L.lt_naive_workspace_bytes.restype = C.c_size_t
            L.lt_backward_lrb2.argtypes = [V, P(lt_params), P(lt_render_opts), V, V, C.c_size_t, P(lt_grads), V]
            L.lt_lrb2_buffer_bytes.argtypes = [P(lt_render_opts)]
            L.lt_lrb2_buffer_bytes.restype = C.c_size_t
            L.lt_lrb3_state_bytes.argtypes = [P(lt_render_opts)]
            L.lt_lrb3_state_bytes.restype = C.c_size_t
            L.lt_bidir_primal.argtypes = [V, P(lt_params), P(lt_render_opts), P(lt_bidir_opts), V, V]
            L.lt_bidir_backward.argtypes = [V, P(lt_params), P(lt_render_opts), P(lt_bidir_opts), V, P(lt_grads), V]
            L.lt_sync_status.argtypes = [V, V]
            L.lt_last_error.restype = C.c_char_p
            L.lt_version.restype = C.c_char_p
            L.lt_mlp_collect.argtypes = [V, P(lt_params), P(lt_render_opts), V, C.c_float, V, V, C.c_int64, V, V]
            L.lt_mlp_init_stats.argtypes = [V, V, V, C.c_int64, V]
            L.lt_mlp_grad.argtypes = [V, V, V, C.c_int64, C.c_int64, V, V, V]
            L.lt_mlp_adam.argtypes = [V, V, V, V, C.c_int, C.c_float, V]
            L.lt_mlp_forward.argtypes = [V, V, C.c_int64, V, V]
            L.lt_batch_create.argtypes = [P(lt_batch_item), C.c_int, V, P(V)]
            L.lt_batch_run.argtypes = [V, C.c_int, V]
            L.lt_batch_set_config.argtypes = [V, P(lt_batch_config)]
            L.lt_batch_get_config.argtypes = [V, P(lt_batch_config)]
            L.lt_batch_tune.argtypes = [V, C.c_int, C.c_int, V, P(lt_batch_config), P(C.c_float)]
            L.lt_batch_destroy.argtypes = [V]
            L.lt_batch_destroy.restype = None
            _lib = L
    return _lib


def _check(status: int):
    if status != LT_OK:
        raise LTError(status, lib().lt_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Scene:
    """A scene on the current CUDA device: geometry + BVH in liblt, parameters as torch tensors."""

    def __init__(self, sc: "_inputs.Scene", device=None, stream=None):
        if not torch.cuda.is_available():
            raise LTError(LT_ERR_UNSUPPORTED, "liblt needs a CUDA device")
        self.src = sc
        self.device = torch.device(device or "cuda")
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        d = lt_scene_desc()
        d.n_quads = sc.n_quads
        d.quads = arr(sc.quads.reshape(-1), np.float32)
        d.n_verts = int(sc.verts.shape[0])
        d.verts = arr(sc.verts.reshape(-1), np.float32) if sc.verts.size else None
        d.vert_h = arr(sc.vert_h, np.int32) if sc.vert_h.size else None
        d.n_tris = sc.n_tris
        d.tris = arr(sc.tris.reshape(-1), np.int32) if sc.tris.size else None
        d.prim_mat = arr(sc.prim_mat, np.int32)
        d.n_mats = int(sc.mat_type.size)
        d.mat_type = arr(sc.mat_type, np.int32)
        d.mat_ior = arr(sc.mat_ior, np.float32)
        d.mat_tex_off = arr(sc.mat_tex_off, np.int32)
        d.mat_tex_w = arr(sc.mat_tex_w, np.int32)
        d.mat_tex_h = arr(sc.mat_tex_h, np.int32)
        d.emitter_quad = sc.emitter_quad
        d.cam_pos = F3(*sc.cam_pos)
        d.cam_look = F3(*sc.cam_look)
        d.cam_up = F3(*sc.cam_up)
        d.fov_y_deg = sc.fov_y_deg
        d.width, d.height = sc.W, sc.H
        d.n_albedo = int(sc.albedo.size)
        d.n_heights = int(sc.heights.size)
        self.W, self.H = sc.W, sc.H
        self.n_albedo, self.n_heights = d.n_albedo, d.n_heights
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().lt_scene_create(C.byref(d), _stream(stream), C.byref(h)))
        self._h = h
        f32 = dict(device=self.device, dtype=torch.float32)
        self.albedo = torch.tensor(sc.albedo, **f32) if sc.albedo.size else torch.zeros(1, **f32)
        self.Le = torch.tensor(sc.Le, **f32)
        self.heights = torch.tensor(sc.heights, **f32) if sc.heights.size else torch.zeros(1, **f32)
        if self.n_heights:
            self.refit(self.heights, stream)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            try:
                torch.cuda.synchronize(self.device)
            except Exception:
                pass
            _lib.lt_scene_destroy(h)
            self._h = None

    # ------------------------------------------------------------------ calls
    def refit(self, heights, stream=None):
        heights = heights.contiguous()
        self.heights = heights
        _check(lib().lt_scene_refit(self._h, _ptr(heights), _stream(stream)))

    def params(self, albedo=None, Le=None):
        a = (albedo if albedo is not None else self.albedo).contiguous()
        le = (Le if Le is not None else self.Le).contiguous()
        self._keep_params = (a, le)
        return lt_params(a.data_ptr(), le.data_ptr())

    @staticmethod
    def opts(seed=0, n_paths=1 << 14, max_depth=4, attached=0, path_offset=0, n_norm=0, block_size=0,
             blocks_per_sm=0, mask=None, hash_out=None, dbg_out=None, target=TARGET_LUMINANCE, mlp=None,
             census=None, lrb3_state=None, lrb3_mask_ready=0, bvh_width=0, rr_depth=0, rr_prob=1.0, filter=0,
             scatter=0, literal=0, jac_noise=0, noise_seed=0, det_eps=0.0):
        """Render options.  `lrb3_state`: a device buffer of lrb3_state_bytes(opts) bytes
        selects the separate-pass form of lt_backward_lrb3, and a plain primal given it stores
        the paths' connection-validity masks, the list of paths with a connection and each
        path's first connection there; `lrb3_mask_ready=1` lets the backward reuse them (see
        include/lt.h)."""
        o = lt_render_opts()
        o.seed, o.path_offset, o.n_paths, o.n_norm = int(seed), int(path_offset), int(n_paths), int(n_norm)
        o.max_depth, o.attached, o.target = int(max_depth), int(attached), int(target)
        o.mlp = None if mlp is None else mlp.data_ptr()
        o.block_size, o.blocks_per_sm = int(block_size), int(blocks_per_sm)
        o.path_mask = None if mask is None else mask.data_ptr()
        o.path_hash = None if hash_out is None else hash_out.data_ptr()
        o.path_dbg = None if dbg_out is None else dbg_out.data_ptr()
        o.census = None if census is None else census.data_ptr()
        o.bvh_width = int(bvh_width)
        o.scatter = int(scatter)
        o.literal, o.jac_noise, o.noise_seed, o.det_eps = int(literal), int(jac_noise), int(noise_seed), float(det_eps)
        o.rr_depth, o.rr_prob, o.filter = int(rr_depth), float(rr_prob), int(filter)
        o.lrb3_mask_ready = int(lrb3_mask_ready)
        o.lrb3_state = None if lrb3_state is None else lrb3_state.data_ptr()
        o.lrb3_state_bytes = 0 if lrb3_state is None else lrb3_state.numel() * lrb3_state.element_size()
        # the struct holds raw device pointers: keep the tensors alive as long as it lives
        o._keep = (mask, hash_out, dbg_out, census, mlp, lrb3_state)
        return o

    @staticmethod
    def lrb3_state_bytes(n_paths) -> int:
        o = lt_render_opts()
        o.n_paths = int(n_paths)
        return int(lib().lt_lrb3_state_bytes(C.byref(o)))

    def new_lrb3_state(self, n_paths):
        return torch.empty(self.lrb3_state_bytes(n_paths), dtype=torch.uint8, device=self.device)

    def record_size(self, o) -> int:
        return int(lib().lt_record_size(C.byref(o)))

    def naive_workspace_bytes(self, o) -> int:
        return int(lib().lt_naive_workspace_bytes(C.byref(o)))

    def lrb2_buffer_bytes(self, o) -> int:
        return int(lib().lt_lrb2_buffer_bytes(C.byref(o)))

    def new_image(self):
        return torch.empty((self.H, self.W, 3), device=self.device, dtype=torch.float32)

    def primal(self, o, estimator=EST_PLAIN, image=None, aux=None, albedo=None, Le=None, stream=None):
        img = image if image is not None else self.new_image()
        p = self.params(albedo, Le)
        nbytes = 0 if aux is None else aux.numel() * aux.element_size()
        _check(lib().lt_primal(self._h, C.byref(p), C.byref(o), int(estimator), _ptr(img), _ptr(aux), nbytes,
                               _stream(stream)))
        return img

    def _grads(self, d_albedo, d_Le, d_heights, accumulate):
        return lt_grads(None if d_albedo is None else d_albedo.data_ptr(), None if d_Le is None else d_Le.data_ptr(),
                        None if d_heights is None else d_heights.data_ptr(), int(accumulate))

    def new_grads(self):
        f32 = dict(device=self.device, dtype=torch.float32)
        return (torch.zeros(max(1, self.n_albedo), **f32), torch.zeros(3, **f32),
                torch.zeros(max(1, self.n_heights), **f32))

    def backward_lrb3(self, o, d_image, grads=None, accumulate=False, albedo=None, Le=None, stream=None):
        g = grads if grads is not None else self.new_grads()
        p = self.params(albedo, Le)
        gr = self._grads(*g, accumulate)
        _check(lib().lt_backward_lrb3(self._h, C.byref(p), C.byref(o), _ptr(d_image.contiguous()), C.byref(gr),
                                      _stream(stream)))
        return g

    def backward_reslrb(self, o, d_image, records, grads=None, accumulate=False, albedo=None, Le=None, stream=None):
        g = grads if grads is not None else self.new_grads()
        p = self.params(albedo, Le)
        gr = self._grads(*g, accumulate)
        _check(lib().lt_backward_reslrb(self._h, C.byref(p), C.byref(o), _ptr(d_image.contiguous()), _ptr(records),
                                        C.byref(gr), _stream(stream)))
        return g

    def backward_lrb2(self, o, d_image, buffer, grads=None, accumulate=False, albedo=None, Le=None, stream=None):
        """Buffered two-pass backward from the buffer lt_primal(EST_BUFFERED) filled."""
        g = grads if grads is not None else self.new_grads()
        p = self.params(albedo, Le)
        gr = self._grads(*g, accumulate)
        nbytes = buffer.numel() * buffer.element_size()
        _check(lib().lt_backward_lrb2(self._h, C.byref(p), C.byref(o), _ptr(d_image.contiguous()), _ptr(buffer),
                                      nbytes, C.byref(gr), _stream(stream)))
        return g

    def backward_naive(self, o, d_image, workspace, grads=None, accumulate=False, albedo=None, Le=None, stream=None):
        g = grads if grads is not None else self.new_grads()
        p = self.params(albedo, Le)
        gr = self._grads(*g, accumulate)
        nbytes = workspace.numel() * workspace.element_size()
        _check(lib().lt_backward_naive(self._h, C.byref(p), C.byref(o), _ptr(d_image.contiguous()), _ptr(workspace),
                                       nbytes, C.byref(gr), _stream(stream)))
        return g

    @staticmethod
    def bidir_opts(n_cam, cam_mask=None, cam_hash=None):
        """Camera-side settings of the bidirectional estimator (see include/lt.h)."""
        b = lt_bidir_opts(int(n_cam), None if cam_mask is None else cam_mask.data_ptr(),
                          None if cam_hash is None else cam_hash.data_ptr())
        b._keep = (cam_mask, cam_hash)
        return b

    def bidir_primal(self, o, b, image=None, albedo=None, Le=None, stream=None):
        """Bidirectional image: light paths of `o` and camera samples of `b` (bidir_opts)."""
        img = image if image is not None else self.new_image()
        p = self.params(albedo, Le)
        _check(lib().lt_bidir_primal(self._h, C.byref(p), C.byref(o), C.byref(b), _ptr(img), _stream(stream)))
        return img

    def bidir_backward(self, o, b, d_image, grads=None, accumulate=False, albedo=None, Le=None, stream=None):
        """Gradient of <d_image, bidirectional image>: LRB-3 on the light paths, path replay
        backpropagation on the camera samples."""
        g = grads if grads is not None else self.new_grads()
        p = self.params(albedo, Le)
        gr = self._grads(*g, accumulate)
        _check(lib().lt_bidir_backward(self._h, C.byref(p), C.byref(o), C.byref(b), _ptr(d_image.contiguous()),
                                       C.byref(gr), _stream(stream)))
        return g

    def mlp_collect(self, o, d_image, capacity, target_floor=0.0, stream=None):
        """Training pairs (features [n,16], targets [n]) from an LRB-3 pass-2 replay."""
        f = torch.empty((capacity, 16), device=self.device, dtype=torch.float32)
        t = torch.empty(capacity, device=self.device, dtype=torch.float32)
        cnt = torch.zeros(1, device=self.device, dtype=torch.int64)
        p = self.params()
        _check(lib().lt_mlp_collect(self._h, C.byref(p), C.byref(o), _ptr(d_image.contiguous()), float(target_floor),
                                    _ptr(f), _ptr(t), int(capacity), _ptr(cnt), _stream(stream)))
        n = min(int(cnt.item()), capacity)
        return f[:n], t[:n], int(cnt.item())

    def sync_status(self, stream=None):
        _check(lib().lt_sync_status(self._h, _stream(stream)))


class Batch:
    """Many scenes in one persistent launch per pass (lt_batch_*).

    `items`: list of dicts with keys scene (Scene), n_paths, max_depth and optionally seed,
    path_offset, n_norm, attached, mask (uint8 per path, 0 = skip), albedo, Le, heights
    (refit by the primal passes),
    d_image, reslrb (allocate ResLRB records), lrb3_state (allocate an LRB-3 state: the
    LRB-3 pass then runs in two kernels reusing the primal pass's validity masks),
    accumulate.  The batch allocates each item's
    image, records and gradients (attributes of the item dicts: image, records, grads) and
    keeps every tensor alive; change parameter values in place (copy_) between runs."""

    def __init__(self, items, stream=None):
        self.items = items
        arr = (lt_batch_item * len(items))()
        for k, it in enumerate(items):
            S = it["scene"]
            it["_state"] = S.new_lrb3_state(it["n_paths"]) if it.get("lrb3_state") else None
            o = Scene.opts(seed=it.get("seed", 0), n_paths=it["n_paths"], max_depth=it["max_depth"],
                           attached=it.get("attached", 0), path_offset=it.get("path_offset", 0),
                           n_norm=it.get("n_norm", 0), dbg_out=it.get("dbg_out"), mask=it.get("mask"),
                           lrb3_state=it["_state"], lrb3_mask_ready=int(it["_state"] is not None))
            it.setdefault("albedo", S.albedo)
            it.setdefault("Le", S.Le)
            it.setdefault("d_image", torch.zeros((S.H, S.W, 3), device=S.device))
            it["image"] = S.new_image()
            it["grads"] = S.new_grads()
            it["records"] = (torch.empty((max(1, it["n_paths"]), 8), device=S.device)
                             if it.get("reslrb") else None)
            it["_opts"] = o
            e = arr[k]
            e.scene = S._h.value
            e.params = lt_params(it["albedo"].data_ptr(), it["Le"].data_ptr())
            h = it.get("heights")
            e.heights = None if h is None else h.data_ptr()
            e.opts = o
            e.image = it["image"].data_ptr()
            e.records = None if it["records"] is None else it["records"].data_ptr()
            e.d_image = it["d_image"].data_ptr()
            e.grads = S._grads(*it["grads"], it.get("accumulate", False))
        h = C.c_void_p()
        _check(lib().lt_batch_create(arr, len(items), _stream(stream), C.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            try:
                torch.cuda.synchronize()
            except Exception:
                pass
            _lib.lt_batch_destroy(h)
            self._h = None

    def run(self, pass_id, stream=None):
        _check(lib().lt_batch_run(self._h, int(pass_id), _stream(stream)))

    @staticmethod
    def _cfg(c):
        return dict(block_size=c.block_size, paths_per_thread=c.paths_per_thread, blocks_per_sm=c.blocks_per_sm,
                    bvh_width=c.bvh_width)

    def config(self):
        c = lt_batch_config()
        _check(lib().lt_batch_get_config(self._h, C.byref(c)))
        return self._cfg(c)

    def set_config(self, block_size=128, paths_per_thread=4, blocks_per_sm=0, bvh_width=4):
        c = lt_batch_config(int(block_size), int(paths_per_thread), int(blocks_per_sm), int(bvh_width))
        _check(lib().lt_batch_set_config(self._h, C.byref(c)))

    def tune(self, pass_id, reps=2, stream=None):
        """Autotune block size x paths per thread x BVH width for `pass_id`; returns
        (config, ms)."""
        c = lt_batch_config()
        ms = C.c_float()
        _check(lib().lt_batch_tune(self._h, int(pass_id), int(reps), _stream(stream), C.byref(c), C.byref(ms)))
        return self._cfg(c), float(ms.value)


def film_l2(image, target, d_image=None, loss=None, stream=None):
    """L2 film loss and its image adjoint (lt_film_l2)."""
    d = d_image if d_image is not None else torch.empty_like(image)
    l = loss if loss is not None else torch.empty(1, device=image.device, dtype=torch.float32)
    _check(lib().lt_film_l2(_ptr(image.contiguous()), _ptr(target.contiguous()), image.numel(), _ptr(d), _ptr(l),
                            _stream(stream)))
    return l, d


def version() -> str:
    return lib().lt_version().decode()


# ------------------------------------------------------------------ learned reservoir target
def mlp_init(seed=0, device="cuda"):
    """Fresh parameter block (He-initialised weights, zero biases, identity statistics)."""
    g = torch.Generator().manual_seed(seed)
    P = torch.zeros(MLP_PARAMS, dtype=torch.float32)
    P[0:1024] = torch.randn(1024, generator=g) * (2.0 / 16) ** 0.5
    P[1088:5184] = torch.randn(4096, generator=g) * (2.0 / 64) ** 0.5
    P[5248:5312] = torch.randn(64, generator=g) * (1.0 / 64) ** 0.5
    P[5329:5345] = 1.0  # 1/std
    P[5345] = 1.0       # target scale
    return P.to(device)


def mlp_init_stats(P, feats, targets, stream=None):
    _check(lib().lt_mlp_init_stats(_ptr(P), _ptr(feats.contiguous()), _ptr(targets.contiguous()), feats.shape[0],
                                   _stream(stream)))


def mlp_grad(P, feats, targets, grad, loss, batch=None, stream=None):
    n = feats.shape[0]
    _check(lib().lt_mlp_grad(_ptr(P), _ptr(feats.contiguous()), _ptr(targets.contiguous()), n, int(batch or n),
                             _ptr(grad), _ptr(loss), _stream(stream)))


def mlp_adam(P, m, v, grad, step, lr, stream=None):
    _check(lib().lt_mlp_adam(_ptr(P), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr), _stream(stream)))


def mlp_forward(P, feats, out=None, stream=None):
    o = out if out is not None else torch.empty(feats.shape[0], device=feats.device, dtype=torch.float32)
    _check(lib().lt_mlp_forward(_ptr(P), _ptr(feats.contiguous()), feats.shape[0], _ptr(o), _stream(stream)))
    return o


def mlp_train(P, feats, targets, epochs=20, batch=4096, lr=1e-3, seed=0, stream=None):
    """Adam on the standardized-target MSE with the project's tensor-core kernels; returns
    the per-epoch mean losses.  (Mini-batches are contiguous slices of a seeded permutation.)"""
    n = feats.shape[0]
    mlp_init_stats(P, feats, targets, stream)
    m = torch.zeros(MLP_WEIGHTS, device=P.device)
    v = torch.zeros(MLP_WEIGHTS, device=P.device)
    grad = torch.zeros(MLP_WEIGHTS, device=P.device)
    loss = torch.zeros(1, device=P.device)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses, step = [], 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(P.device)
        fx, tx = feats[perm].contiguous(), targets[perm].contiguous()
        loss.zero_()
        nb = 0
        for b0 in range(0, n, batch):
            b1 = min(n, b0 + batch)
            grad.zero_()
            mlp_grad(P, fx[b0:b1], tx[b0:b1], grad, loss, batch=b1 - b0, stream=stream)
            step += 1
            mlp_adam(P, m, v, grad, step, lr, stream=stream)
            nb += 1
        losses.append(float(loss.item()) / nb)
    return losses
