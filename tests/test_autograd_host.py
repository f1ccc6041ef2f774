"""Host logic of the autograd wrapper (CPU, no kernels): a stand-in scene records what the
wrapper asks of it, so these tests check the order of calls and the arguments — the
geometry each backward replays against, the LRB-3 state it hands over, the gradients it
returns — not the arithmetic, which the GPU tests check against the oracle."""
from types import SimpleNamespace

import pytest
import torch

from paper_2609_32920_gb300 import autograd as A


class StandInScene:
    """Records refits and hands out distinct per-render buffers; its 'image' and
    'gradients' are tagged with the heights the scene holds when they are computed."""
    device = "cpu"
    W, H = 2, 2

    def __init__(self, n_heights=3):
        self.n_heights = n_heights
        self.h = torch.zeros(n_heights)
        self.states = []
        self.calls = []

    def refit(self, h):
        self.h = h.clone()
        self.calls.append("refit")

    def new_lrb3_state(self, n):
        st = torch.zeros(4)
        self.states.append(st)
        return st

    def opts(self, **kw):
        kw.setdefault("lrb3_state", None)
        kw.setdefault("lrb3_mask_ready", 0)
        return SimpleNamespace(**kw)

    def naive_workspace_bytes(self, o):
        return 16

    def lrb2_buffer_bytes(self, o):
        return 16

    def primal(self, o, estimator, aux, albedo, Le):
        self.calls.append(("primal", estimator))
        return torch.full((self.H, self.W, 3), float(self.h.sum()))

    def _grads(self, o, gI, albedo, Le, method, aux=None):
        self.calls.append((method, o.lrb3_state, o.lrb3_mask_ready, aux))
        tag = float(self.h.sum())
        return (torch.full((albedo.numel() + 5,), tag), torch.full((3,), tag),
                torch.full((max(self.n_heights, 1) + 7,), tag))

    def backward_lrb3(self, o, gI, albedo, Le):
        return self._grads(o, gI, albedo, Le, "lrb3")

    def backward_reslrb(self, o, gI, rec, albedo, Le):
        return self._grads(o, gI, albedo, Le, "reslrb", rec)

    def backward_naive(self, o, gI, ws, albedo, Le):
        return self._grads(o, gI, albedo, Le, "naive", ws)

    def backward_lrb2(self, o, gI, buf, albedo, Le):
        return self._grads(o, gI, albedo, Le, "lrb2", buf)


def _params(n_heights=3, h=0.0):
    albedo = torch.rand(6, requires_grad=True)
    Le = torch.ones(3, requires_grad=True)
    heights = torch.full((n_heights,), h, requires_grad=True)
    return albedo, Le, heights


@pytest.mark.parametrize("method", A.METHODS)
def test_each_backward_replays_against_its_own_forward_geometry(method):
    """Two renders of one scene at different heights, then both backwards (in reverse
    order): each gradient is computed with the scene refitted to its own render's heights."""
    S = StandInScene()
    a1, L1, h1 = _params(h=1.0)
    a2, L2, h2 = _params(h=2.0)
    img1 = A.render(S, a1, L1, h1, method=method, n_paths=8)
    img2 = A.render(S, a2, L2, h2, method=method, n_paths=8)
    assert float(img1[0, 0, 0].detach()) == pytest.approx(3.0) and float(img2[0, 0, 0].detach()) == pytest.approx(6.0)
    img2.sum().backward()
    img1.sum().backward()
    for (a, L, h), tag in (((a1, L1, h1), 3.0), ((a2, L2, h2), 6.0)):
        assert a.grad.shape == a.shape and L.grad.shape == L.shape and h.grad.shape == h.shape
        assert torch.all(h.grad == tag) and torch.all(a.grad == tag) and torch.all(L.grad == tag)
    # the scene is left at the heights of the last backward's render
    assert torch.equal(S.h, h1.detach())


def test_lrb3_backward_takes_the_state_its_forward_filled():
    S = StandInScene()
    a1, L1, h1 = _params(h=1.0)
    a2, L2, h2 = _params(h=2.0)
    img1 = A.render(S, a1, L1, h1, method="lrb3", n_paths=8)
    img2 = A.render(S, a2, L2, h2, method="lrb3", n_paths=8)
    img1.sum().backward()
    img2.sum().backward()
    bw = [c for c in S.calls if isinstance(c, tuple) and c[0] == "lrb3"]
    assert len(S.states) == 2 and len(bw) == 2
    assert bw[0][1] is S.states[0] and bw[1][1] is S.states[1]
    assert bw[0][2] == 1 and bw[1][2] == 1  # the primal's masks are reused


def test_gradients_only_for_inputs_that_require_them():
    S = StandInScene()
    albedo = torch.rand(6, requires_grad=True)
    Le = torch.ones(3)
    heights = torch.zeros(3)
    A.render(S, albedo, Le, heights, method="naive", n_paths=8).sum().backward()
    assert albedo.grad is not None and Le.grad is None and heights.grad is None


def test_scene_without_heights_is_never_refitted():
    S = StandInScene(n_heights=0)
    albedo, Le, heights = _params(n_heights=0)
    A.render(S, albedo, Le, heights, method="reslrb", n_paths=8).sum().backward()
    assert "refit" not in S.calls
    assert albedo.grad is not None and heights.grad.shape == (0,)


def test_unknown_method_is_rejected():
    S = StandInScene()
    with pytest.raises(ValueError):
        A.render(S, *_params(), method="ptracer")
