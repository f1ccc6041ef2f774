"""The allocation-free naive-AD gradient (lt_naive_gradient_static) against the existing
two calls with a caller workspace (lt_primal(LT_EST_NAIVE) + lt_backward_naive).

This entry point is for callers that cannot allocate GPU memory while they run (a fixed
memory budget, or a loop that must never trigger the device-wide synchronisation that
cudaMalloc/cudaFree can cause): its tape lives in a fixed array compiled into the
library.  The file is named so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2609_32920_gb300 import inputs as I
from paper_2609_32920_gb300 import lt
from tests.gpu_util import primal_close, rel_l2, t32

pytestmark = pytest.mark.gpu

LT_NAIVE_STATIC_BYTES = 32 << 20


def _static_call(S, o, dI, image, grads):
    L = lt.lib()
    fn = L.lt_naive_gradient_static
    fn.argtypes = [C.c_void_p, C.POINTER(lt.lt_params), C.POINTER(lt.lt_render_opts), C.c_void_p, C.c_void_p,
                   C.POINTER(lt.lt_grads), C.c_void_p]
    p = S.params()
    g = lt.lt_grads(grads[0].data_ptr(), grads[1].data_ptr(), grads[2].data_ptr(), 0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(S._h, C.byref(p), C.byref(o), C.c_void_p(dI.data_ptr()), C.c_void_p(image.data_ptr()), C.byref(g),
              stream)


@pytest.mark.parametrize("attached", [0, 1])
def test_static_tape_gradient_matches_workspace_calls_twice_in_a_row(attached):
    sc = I.box_scene(32, heightmap=6, hm_std=0.03)
    S = lt.Scene(sc)
    dI = t32(I.smooth_adjoint(sc.W, sc.H, 91))
    # two calls in a row share (and overwrite) the fixed tape; the second is smaller, so its
    # tape layout (header size, depth stride) differs and stale entries of the first remain
    for seed, n, D in ((5, 3000, 7), (6, 1200, 4)):
        o = S.opts(seed=seed, n_paths=n, max_depth=D, attached=attached)
        assert S.naive_workspace_bytes(o) <= LT_NAIVE_STATIC_BYTES
        ws = torch.empty(S.naive_workspace_bytes(o), dtype=torch.uint8, device="cuda")
        ref_img = S.primal(o, estimator=lt.EST_NAIVE, aux=ws).clone()
        ref_g = [x.clone() for x in S.backward_naive(o, dI, ws)]
        img = S.new_image()
        grads = S.new_grads()
        assert _static_call(S, o, dI, img, grads) == lt.LT_OK, lt.lib().lt_last_error()
        torch.cuda.synchronize()
        a, b = img.cpu().numpy(), ref_img.cpu().numpy()
        assert primal_close(a, b).all()
        for x, y in zip(grads, ref_g):
            assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-3
        assert np.abs(ref_g[0].cpu().numpy()).sum() > 0
    S.sync_status()


def test_static_tape_rejects_requests_beyond_its_size():
    sc = I.box_scene(16)
    S = lt.Scene(sc)
    dI = torch.zeros((16, 16, 3), device="cuda")
    o = S.opts(seed=0, n_paths=1 << 20, max_depth=16)  # 512 MiB of tape
    assert S.naive_workspace_bytes(o) > LT_NAIVE_STATIC_BYTES
    img = S.new_image()
    grads = S.new_grads()
    assert _static_call(S, o, dI, img, grads) == lt.LT_ERR_INVALID_ARG
    assert b"fixed scratch" in lt.lib().lt_last_error()
    # a path count whose byte size would wrap around is rejected as well
    o = S.opts(seed=0, n_paths=1 << 62, max_depth=64)
    assert _static_call(S, o, dI, img, grads) == lt.LT_ERR_INVALID_ARG
