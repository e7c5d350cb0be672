"""Multi-process host logic on CPU (gloo, world size 2): the instance partition of a
batch, the whole-job throughput (units of all ranks over the slowest rank's time) and the
sharded batch itself: the instances a rank draws are bit-identical to the same instances
of the unsharded batch (every instance is seeded by its own id)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2106_11594_gb300 import dist as rgdist
from paper_2106_11594_gb300 import inputs


# small uneven shapes (n, m, r) for the sharded-batch identity check
SMALL_SHAPES = [(40 + 7 * b, 8 + (5 * b) % 29, 2 + b % 5) for b in range(13)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, m, r = inputs.uneven_batch_shapes(256)
        parts = rgdist.lpt_partition(rgdist.instance_cost(n, m, r), world)
        mine = parts[rank]
        # every rank derives the same partition; gather the other ranks' views
        flat = torch.tensor(np.concatenate(parts), dtype=torch.int64)
        views = [torch.empty_like(flat) for _ in range(world)]
        dist.all_gather(views, flat)
        same = all(bool(torch.equal(v, flat)) for v in views)
        rows_mine = float(n[mine].sum())
        ms_mine = 10.0 + 5.0 * rank  # rank 1 is the slower one
        rate, ms, units = rgdist.job_throughput(rows_mine, ms_mine)
        # the bench's sharded batch: this rank's share, drawn on its own, equals the same
        # instances cut out of the whole batch, bit for bit
        import bench
        cpu = torch.device("cpu")
        bat = bench.BatchOnGpu(SMALL_SHAPES, 3, 1e-4, cpu, world, rank)
        full = bench.BatchOnGpu(SMALL_SHAPES, 3, 1e-4, cpu, 1, 0)
        ident = True
        for k, i in enumerate(bat.ids):
            ident &= torch.equal(bat.A[bat.eo[k]:bat.eo[k + 1]], full.A[full.eo[i]:full.eo[i + 1]])
            ident &= torch.equal(bat.Y[bat.ro[k]:bat.ro[k + 1]], full.Y[full.ro[i]:full.ro[i + 1]])
        cover = torch.zeros(len(SMALL_SHAPES), dtype=torch.int64)
        cover[torch.tensor(bat.ids, dtype=torch.int64)] = 1
        dist.all_reduce(cover)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([rate, ms, units, float(same), float(len(mine)), float(ident),
                          float((cover == 1).all()), float(len(bat.ids))]))
    finally:
        dist.destroy_process_group()


def test_lpt_partition_is_a_balanced_partition():
    n, m, r = inputs.uneven_batch_shapes(4096)
    c = rgdist.instance_cost(n, m, r)
    for world in (1, 2, 3, 8):
        parts = rgdist.lpt_partition(c, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(c)))
        loads = np.array([c[p].sum() for p in parts])
        # LPT bound: max load <= mean + max single cost
        assert loads.max() <= loads.mean() + c.max() + 1e-6


def test_lpt_partition_small_cases():
    assert [p.tolist() for p in rgdist.lpt_partition([5, 1, 4], 2)] == [[0], [1, 2]]
    assert [p.tolist() for p in rgdist.lpt_partition([], 2)] == [[], []]
    with pytest.raises(ValueError):
        rgdist.lpt_partition([1.0], 0)


def test_job_throughput_without_process_group():
    rate, ms, units = rgdist.job_throughput(1000.0, 2.0)
    assert (rate, ms, units) == (500000.0, 2.0, 1000.0)


def test_gloo_two_ranks(tmp_path):
    world = 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"r{k}.npy") for k in range(world)]
    n, m, r = inputs.uneven_batch_shapes(256)
    total_rows = float(n.sum())
    for v in res:
        rate, ms, units, same, cnt, ident, cover, nb = v
        assert same == 1.0
        assert ident == 1.0  # a rank's instances equal the unsharded batch's
        assert cover == 1.0  # every instance on exactly one rank
        assert 0 < nb < len(SMALL_SHAPES)
        assert ms == 15.0  # the slowest rank's time
        assert units == total_rows  # every instance counted once
        assert rate == pytest.approx(total_rows / 0.015)
    assert res[0][4] + res[1][4] == 256
