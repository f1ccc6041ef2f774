"""Multi-rank path: two gloo ranks on CPU trace disjoint path ranges (the oracle stands in
for the GPU kernels); their images and gradients sum to the single-process ones and the
benchmark's max-over-ranks timing reduction agrees."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_32920_gb300.shard import max_over_ranks, path_shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2609_32920_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = I.box_scene(16)
    off, n, norm = path_shard(rank, world, 3000)
    img = O.render(sc, seed=4, n_paths=n, path_begin=off, n_norm=norm, max_depth=4, n_threads=2)
    g = O.gradient(sc, I.smooth_adjoint(sc.W, sc.H, 3), seed=4, n_paths=n, path_begin=off, n_norm=norm,
                   max_depth=4, n_threads=2)
    t = max_over_ranks(10.0 + rank)
    out[rank] = (img, t, g["d_albedo"], g["d_Le"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_cover_the_single_process_run(oracle):
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    total = res[0][0] + res[1][0]
    from paper_2609_32920_gb300 import inputs as I
    full = oracle.render(I.box_scene(16), seed=4, n_paths=6000, max_depth=4, n_threads=2)
    assert np.allclose(total, full, rtol=1e-12, atol=1e-15)
    sc = I.box_scene(16)
    gfull = oracle.gradient(sc, I.smooth_adjoint(sc.W, sc.H, 3), seed=4, n_paths=6000, max_depth=4, n_threads=2)
    assert np.allclose(res[0][2] + res[1][2], gfull["d_albedo"], rtol=1e-10, atol=1e-14)
    assert np.allclose(res[0][3] + res[1][3], gfull["d_Le"], rtol=1e-10)
    assert res[0][1] == res[1][1] == 11.0
    assert path_shard(1, 2, 3000) == (3000, 3000, 6000)
    with pytest.raises(ValueError):
        path_shard(2, 2, 10)
