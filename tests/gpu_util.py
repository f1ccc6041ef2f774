"""Helpers for the GPU parity tests: run liblt and the oracle on the same seeded inputs,
exclude the rare paths whose discrete decisions differ between FP32 and FP64 (compared
through per-path decision hashes), and compare."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2609_32920_gb300 import lt


def t32(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def rel_l2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def gpu_hashes(S, seed, n, D, **kw):
    h = torch.zeros(n, dtype=torch.int32, device="cuda")
    S.primal(S.opts(seed=seed, n_paths=n, max_depth=D, hash_out=h, **kw))
    torch.cuda.synchronize()
    return h.cpu().numpy().view(np.uint32)


def agree_mask(S, sc, seed, n, D, path_offset=0, n_norm=0, max_divergent=1e-3):
    """Decision-hash agreement between GPU and oracle; returns a uint8 mask."""
    g = gpu_hashes(S, seed, n, D, path_offset=path_offset, n_norm=n_norm)
    _, o = O.render(sc, seed=seed, n_paths=n, max_depth=D, path_begin=path_offset, n_norm=n_norm, want_hash=True)
    same = g == o
    frac = 1.0 - same.mean()
    assert frac <= max_divergent, f"{(~same).sum()} of {n} paths took different discrete decisions"
    return same.astype(np.uint8)


def primal_close(a, b, rtol=1e-4, mass=None, W=None, depth=1):
    """Per pixel |a-b| <= rtol * max(|b|, 1e-3 mean|b|) + eps_u * mass.

    The second term is the FP32 rounding of film positions: u = W/2 (1 + p_x / tan_x) comes
    from the hit point through about ten FP32 operations, so |du| <= 16 * 2^-24 * max(W, H)
    pixels per vertex; each vertex is found from its predecessor (the ray leaves the previous
    vertex, Eq. 2), so the position error can grow along the path, at worst linearly in its
    length `depth`.  A tent tap's weight moves by at most |du|, so a pixel moves by at
    most |du| times its tap mass (sum of |L| over splats touching it, from the oracle).  A
    splat within rounding of a pixel-centre line may use a tap set shifted by one pixel
    (with a near-zero weight there), so the mass is dilated over each pixel's 3x3
    neighbourhood."""
    a, b = np.asarray(a), np.asarray(b)
    floor = 1e-3 * np.abs(b).mean()
    tol = rtol * np.maximum(np.abs(b), floor)
    if mass is not None:
        m = np.asarray(mass)
        pad = np.pad(m, ((1, 1), (1, 1), (0, 0)))
        dil = np.max([pad[i:i + m.shape[0], j:j + m.shape[1]] for i in range(3) for j in range(3)], axis=0)
        tol = tol + 16.0 * 2.0 ** -24 * float(W) * float(depth) * dil
    return np.abs(a - b) <= tol
