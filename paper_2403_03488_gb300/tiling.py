"""One large image shared by several ranks (one GPU each): row strips with a
halo exchanged between neighbouring ranks.

A BM3D output pixel depends only on the noisy pixels within the halo radius
of it (dn_bm3d_halo: the search-window reach of both passes), so a rank that
holds rows [r0, r1) of the image and receives `halo` rows above and below
from its neighbours computes rows [r0, r1) of the whole-image result exactly,
provided r0 and the halo lie on the reference grids of both passes (multiples
of the steps' least common multiple).  The exchange is the only
communication: point-to-point sends of boundary rows to the neighbouring
ranks (torch.distributed: gloo on CPU tensors, NCCL on device tensors).
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Tuple

import torch
import torch.distributed as dist


def grid_multiple(params) -> int:
    """Least common multiple of the two passes' reference grid steps."""
    return math.lcm(int(params.hard.step), int(params.wiener.step))


def halo_rows(radius: int, g: int) -> int:
    """The dependency radius rounded up to a multiple of g."""
    return -(-int(radius) // g) * g


def strip_rows(H: int, world: int, g: int) -> List[Tuple[int, int]]:
    """Row ranges [r0, r1) of the ranks' strips: as equal as the grid multiple
    g allows, every boundary a multiple of g."""
    units = -(-H // g)
    out, u0 = [], 0
    for r in range(world):
        u1 = u0 + units // world + (1 if r < units % world else 0)
        out.append((min(H, u0 * g), min(H, u1 * g)))
        u0 = u1
    return out


def exchange_halo(strip: torch.Tensor, halo: int, rank: int, world: int,
                  group: Optional[dist.ProcessGroup] = None) -> Tuple[torch.Tensor, int]:
    """strip: [C, h, W], this rank's rows.  Sends its first `halo` rows to
    rank - 1 and its last `halo` rows to rank + 1, receives theirs, and
    returns ([C, top + h + bottom, W], top): the strip extended by the
    neighbours' rows (top = 0 on the first rank, bottom = 0 on the last).
    Every strip but the last must hold at least `halo` rows, so that one hop
    suffices."""
    C, h, W = strip.shape
    if world > 1 and h < halo and rank < world - 1:
        raise ValueError("strip of %d rows is thinner than the halo (%d)" % (h, halo))
    top = min(halo, 0 if rank == 0 else halo)
    bot = 0 if rank == world - 1 else halo
    up = torch.empty((C, top, W), dtype=strip.dtype, device=strip.device)
    down = torch.empty((C, bot, W), dtype=strip.dtype, device=strip.device)
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(strip[:, :halo].contiguous(), rank - 1, group=group))
        reqs.append(dist.irecv(up, rank - 1, group=group))
    if rank < world - 1:
        reqs.append(dist.isend(strip[:, h - min(h, halo):].contiguous(), rank + 1, group=group))
        reqs.append(dist.irecv(down, rank + 1, group=group))
    for r in reqs:
        r.wait()
    return torch.cat([up, strip, down], dim=1), top


def denoise_sharded(strip: torch.Tensor, sigma: float, rank: int, world: int, params=None,
                    denoise: Optional[Callable[[torch.Tensor], torch.Tensor]] = None,
                    group: Optional[dist.ProcessGroup] = None) -> torch.Tensor:
    """Rows [r0, r1) of the whole-image BM3D result from this rank's rows
    [r0, r1) (strip: [C, h, W], r0 on the grid multiple): exchanges the halo
    with the neighbouring ranks, denoises the extended strip on this rank's
    device (denoise_bm3d by default) and keeps its own rows."""
    from . import api
    p = params or api.default_bm3d_params()
    halo = halo_rows(api.bm3d_halo(p), grid_multiple(p))
    ext, top = exchange_halo(strip, halo, rank, world, group)
    if denoise is None:
        out = api.denoise_bm3d(ext.unsqueeze(0).contiguous(), sigma, p)[0]
    else:
        out = denoise(ext)
    return out[:, top:top + strip.shape[1]]
