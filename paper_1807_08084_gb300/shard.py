"""Host-side logic for running the path on several GPUs, one process per GPU.

Pixels are independent units, so the path shards without a data-path
collective:

* per-pixel inverse/det (zinv_det, chol_zinv_det, zinv_det_bwd): any split of
  the pixels; the benchmark gives each rank its own image of the same size
  (weak scaling, `rank_seed`);
* window kernels (multilook_zinv_det, wishart_stat_*): contiguous row blocks
  (`row_block`), each rank reading a halo of r = (win-1)/2 rows from its own copy
  of the input (`halo_block`), so no halo exchange is needed;
* the Wishart loss and weight gradient: per-rank partial sums combined by one
  all-reduce of win*win + 1 values (`sum_over_ranks`).

Timing takes the maximum over ranks (`max_over_ranks`).  Everything here works
with any torch.distributed backend (gloo on CPU in the tests, NCCL on GPUs).
"""
from __future__ import annotations

import torch


def row_block(H: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [y0, y1) of rank `rank` in a balanced contiguous split of H rows."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(H, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def halo_block(H: int, y0: int, y1: int, r: int) -> tuple[int, int]:
    """Input rows a rank reads to produce output rows [y0, y1) with a window of
    radius r: the block plus r rows each side, cut at the image border (where
    the kernels clamp)."""
    return max(0, y0 - r), min(H, y1 + r)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s synthetic image (weak scaling: same size, own data)."""
    return seed + 1000 * rank


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(x: float, device: torch.device | str = "cpu") -> float:
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(t: torch.Tensor) -> torch.Tensor:
    """In-place all-reduce (sum) of a small tensor, e.g. the weight gradient and loss."""
    dist = _dist()
    if dist is not None and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def barrier():
    dist = _dist()
    if dist is not None and dist.get_world_size() > 1:
        dist.barrier()
