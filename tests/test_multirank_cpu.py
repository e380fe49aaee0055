"""The multi-rank host logic of the benchmark on CPU: two processes joined by
a gloo process group (127.0.0.1), as torchrun starts them on a multi-GPU node.
The data path has no collective (each rank denoises its own images); what is
checked is the part that does cross ranks: disjoint image seeds per rank,
the max-over-ranks step time and the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2403_03488_gb300 import synth
        seeds = bench.rank_seeds(rank, batch=3)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        # the slowest rank's time is the job's time
        t = bench.max_over_ranks(10.0 + 5.0 * rank)
        # each rank's images are its own: the first rows of image 0 differ between ranks
        _, noisy = synth.make_batch(seeds[:1], 16, 16, 25.0)
        rows = [None] * world
        dist.all_gather_object(rows, noisy[0, 0, 0].tolist())
        out.put((rank, gathered, t, rows))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_images_and_reduce_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t, rows in res:
        s0, s1 = set(gathered[0]), set(gathered[1])
        assert len(s0) == len(s1) == 3 and not (s0 & s1)
        assert t == 15.0
        assert rows[0] != rows[1]


def test_whole_job_value_and_single_process_reduction():
    import bench
    # 2 ranks x 16.78 MPix in 50 ms per step -> 671 MPix/s for the job
    assert abs(bench.whole_job_value(16.777216, 2, 50.0) - 671.08864) < 1e-6
    # without a process group the reduction is the identity
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.rank_seeds(0, batch=2) == [100, 101] and bench.rank_seeds(1, batch=2) == [102, 103]
    # the batch of a profiling run (--batch) is the one the seeds follow
    old = bench.B
    try:
        bench.B = 3
        assert bench.rank_seeds(1) == [103, 104, 105]
    finally:
        bench.B = old
