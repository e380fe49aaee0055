"""The halo of tiled BM3D, pinned on the CPU with the FP64 oracle, and the
halo exchange of one image shared by two gloo ranks.

The library's dependency radius (dn_bm3d_halo, a host function) must be the
exact reach of the method: with it, BM3D of two overlapping tiles of an image
gives the whole-image result in the tiles' interiors (to FP64 rounding), and
one grid step less already changes the result.  With two ranks (gloo,
127.0.0.1) each holding half of the rows, the exchanged strips are the
image's rows and the stitched per-rank results equal the whole-image oracle."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2403_03488_gb300 import synth  # noqa: E402

SEARCH = 9  # small windows keep the oracle fast: radius 2 (2 * 4 + 7) = 30


def _params():
    from paper_2403_03488_gb300 import api
    p = api.default_bm3d_params()
    p.hard.search = SEARCH
    p.wiener.search = SEARCH
    return p


def _oracle_bm3d(oracle, img, sigma):
    hard, wien = oracle.default_passes(sigma)
    hard.search = SEARCH
    wien.search = SEARCH
    return oracle.bm3d(img, sigma, hard=hard, wiener=wien)[1]


def test_halo_formula_from_the_library():
    from paper_2403_03488_gb300 import api, build
    build.build()
    assert api.bm3d_halo() == 2 * (2 * 19 + 7)
    assert api.bm3d_halo(_params()) == 30


def test_tiles_with_the_halo_reproduce_the_whole_image(oracle):
    from paper_2403_03488_gb300 import api, build
    build.build()
    halo = api.bm3d_halo(_params())
    _, noisy = synth.make_batch([3], 40, 160, 25.0)
    y = noisy[0].astype(np.float64)
    whole = _oracle_bm3d(oracle, y, 25.0)
    split = 78  # tile boundary on the grid (multiple of 3)
    errs = []
    for h in (halo, halo - 3):
        a = _oracle_bm3d(oracle, y[:, :, :split + h], 25.0)
        b = _oracle_bm3d(oracle, y[:, :, split - h:], 25.0)
        stitched = np.concatenate([a[:, :, :split], b[:, :, h:]], axis=2)
        errs.append(np.abs(stitched - whole).max())
    assert errs[0] <= 1e-9, errs
    assert errs[1] > 1e-8, errs  # one grid step less changes the result beyond rounding


def test_strip_rows_on_the_grid():
    from paper_2403_03488_gb300 import tiling
    rows = tiling.strip_rows(100, 3, 3)
    assert rows[0][0] == 0 and rows[-1][1] == 100
    assert all(r1 == s0 for (_, r1), (s0, _) in zip(rows, rows[1:]))
    assert all(r0 % 3 == 0 for r0, _ in rows)
    assert tiling.halo_rows(30, 3) == 30 and tiling.halo_rows(31, 3) == 33


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2403_03488_gb300 import tiling
        p = _params()
        _, noisy = synth.make_batch([4], 84, 48, 25.0)
        img = noisy[0].astype(np.float64)
        g = tiling.grid_multiple(p)
        r0, r1 = tiling.strip_rows(img.shape[1], world, g)[rank]
        strip = torch.from_numpy(img[:, r0:r1].copy())
        halo = tiling.halo_rows(30, g)
        ext, top = tiling.exchange_halo(strip, halo, rank, world)
        e0 = r0 - top
        exact = bool(np.array_equal(ext.numpy(), img[:, e0:e0 + ext.shape[1]]))
        out = tiling.denoise_sharded(strip, 25.0, rank, world, params=p,
                                     denoise=lambda x: torch.from_numpy(_oracle_bm3d(oracle, x.numpy(), 25.0)))
        parts = [None] * world
        dist.all_gather_object(parts, (r0, out.numpy()))
        q.put((rank, exact, parts))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halo_and_match_the_whole_image(oracle):
    from paper_2403_03488_gb300 import build
    build.build()
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, noisy = synth.make_batch([4], 84, 48, 25.0)
    whole = _oracle_bm3d(oracle, noisy[0].astype(np.float64), 25.0)
    for rank, exact, parts in res:
        assert exact, "exchanged rows differ from the image's rows (rank %d)" % rank
        stitched = np.concatenate([a for _, a in sorted(parts, key=lambda t: t[0])], axis=1)
        assert stitched.shape == whole.shape
        assert np.abs(stitched - whole).max() <= 1e-9
