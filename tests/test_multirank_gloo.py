"""The multi-rank host path of `bench.py` on CPU: two ranks over gloo.

Under torchrun each rank builds its own copy of the H² matrix and multiplies
its own column shard of the right-hand sides; the ranks share nothing on the
data path (block CG keeps every column's Krylov space apart, Sec. 5.1).  The
only collectives are the timing barrier and the max-reduction of step times.
Here each rank runs the FP64 oracle product on its shard of a small
workload, and the test checks on every rank:
  - the shard is the rank's own (reproducible, distinct from the other's);
  - the shard's product equals the matching columns of the product of the
    whole block (so sharding by columns is exact);
  - max_over_ranks returns the slowest rank's time on every rank, and
    job_gflops counts all ranks' flops over that time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from oracle import h2_oracle as O  # noqa: E402
from workloads import sphere_points  # noqa: E402

N, M, SEED = 1200, 3, 17


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, errq) -> None:
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                          LOCAL_RANK=str(rank))
        assert bench._dist() == (world, rank, rank)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        pts = sphere_points(N, 2)
        H = O.H2Matrix(pts, q=2, leaf_size=64, eta=2.0, sigma=1e-2, length=0.5)
        X = bench.rank_rhs(N, M, SEED, rank)
        assert np.array_equal(X, bench.rank_rhs(N, M, SEED, rank))
        other = bench.rank_rhs(N, M, SEED, 1 - rank)
        assert not np.allclose(X, other)
        Y = O.h2mm(H, 1.0, X)
        # the whole job's block: the shards side by side, in rank order
        full = np.concatenate([bench.rank_rhs(N, M, SEED, r) for r in range(world)], axis=1)
        Yfull = O.h2mm(H, 1.0, full)
        np.testing.assert_allclose(Y, Yfull[:, rank * M:(rank + 1) * M], rtol=1e-13, atol=1e-13)
        # every rank sees the slowest rank's step time; the job rate counts every rank's flops
        dist.barrier()
        my_ms = 10.0 + 5.0 * rank
        slow = bench.max_over_ranks(my_ms, dist, "cpu")
        assert slow == 10.0 + 5.0 * (world - 1)
        flops = float(H.counts()["n"]) * 1e3
        assert bench.job_gflops(flops, slow * 1e-3, world) == pytest.approx(world * flops / (slow * 1e-3) / 1e9)
        assert bench.max_over_ranks(my_ms, None) == my_ms
        dist.barrier()
        dist.destroy_process_group()
    except BaseException as e:  # reported to the parent, which fails the test
        errq.put(f"rank {rank}: {type(e).__name__}: {e}")
        raise


def test_two_ranks_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    errq = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, errq)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    errors = []
    while not errq.empty():
        errors.append(errq.get())
    assert not alive, "a rank did not finish"
    assert not errors, errors
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
