"""The multi-rank path on CPU: two gloo ranks (spawned processes) exercise the
host logic of paper_1807_08084_gb300.shard against the FP64 oracle.

* window kernels shard by row blocks, each rank reading an r-row halo from its
  own copy of the input: the concatenated blocks equal the full image's result;
* the Wishart loss and weight gradient shard the same way and combine with one
  all-reduce of win*win + 1 values;
* timings combine by a max over ranks.
"""
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    import oracle
    from paper_1807_08084_gb300 import shard
    from paper_1807_08084_gb300 import synth as S
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        o = oracle.load()
        # timing: max over ranks
        assert shard.max_over_ranks(rank + 0.5) == world - 0.5
        # multilook by row blocks with a halo, no exchange
        w = S.scaled(S.WORKLOADS["wishart_pair_4k"], 23, 17)
        s1, s2 = w.image(0), w.image(1)
        H = w.H
        win, r = 5, 2
        y0, y1 = shard.row_block(H, rank, world)
        hy0, hy1 = shard.halo_block(H, y0, y1, r)
        part = o.multilook(s1[:, hy0:hy1], win).reshape(9, hy1 - hy0, w.W)[:, y0 - hy0:y1 - hy0]
        full = o.multilook(s1, win).reshape(9, H, w.W)[:, y0:y1]
        np.testing.assert_array_equal(part, full)
        # Wishart loss and gradient: per-rank partial sums, one all-reduce
        wts = np.linspace(0.5, 1.5, win * win) / (win * win)
        _, q = o.wishart_fwd(s1[:, hy0:hy1], s2[:, hy0:hy1], win, wts, want_map=True)
        loss_part = q.reshape(hy1 - hy0, w.W)[y0 - hy0:y1 - hy0].sum()
        g_part = o.wishart_bwd(s1[:, hy0:hy1], s2[:, hy0:hy1], win, wts,
                               rows=(y0 - hy0, y1 - hy0))
        t = torch.from_numpy(np.concatenate([g_part, [loss_part]]))
        shard.sum_over_ranks(t)
        ref_loss = o.wishart_fwd(s1, s2, win, wts)
        ref_g = o.wishart_bwd(s1, s2, win, wts)
        np.testing.assert_allclose(t[:-1].numpy(), ref_g, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(float(t[-1]), ref_loss, rtol=1e-12)
        # weak-scaling replicas get their own data
        assert shard.rank_seed(w.seed, rank) != shard.rank_seed(w.seed, (rank + 1) % world)
        shard.barrier()
    finally:
        dist.destroy_process_group()


def test_row_blocks_partition():
    from paper_1807_08084_gb300 import shard
    for H in (1, 7, 23, 16384):
        for world in (1, 2, 3, 8):
            blocks = [shard.row_block(H, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == H
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    assert shard.halo_block(100, 0, 50, 3) == (0, 53)
    assert shard.halo_block(100, 50, 100, 3) == (47, 100)
    with pytest.raises(ValueError):
        shard.row_block(10, 2, 2)


def test_two_gloo_ranks():
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)
