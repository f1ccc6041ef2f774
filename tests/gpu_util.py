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


def primal_close(a, b, rtol=1e-4):
    """|a-b| <= rtol * max(|b|, 1e-3 mean|b|) elementwise."""
    a, b = np.asarray(a), np.asarray(b)
    floor = 1e-3 * np.abs(b).mean()
    return np.abs(a - b) <= rtol * np.maximum(np.abs(b), floor)
