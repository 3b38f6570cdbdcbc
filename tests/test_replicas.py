"""Multi-process replicas on CPU (torch.distributed, gloo, world size 2): the
ranks draw disjoint realization ranges, the step time is the max over ranks,
and the spectra's mean and covariance merged across ranks equal those of all
fields together."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1406_6072_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        R = 5
        starts = [replicas.realization_start(rank, world, s, R) for s in range(4)]
        gathered = [None] * world
        dist.all_gather_object(gathered, starts)
        ranges = sorted((a, a + R) for st in gathered for a in st)
        for (a0, a1), (b0, _) in zip(ranges, ranges[1:]):
            assert a1 <= b0  # disjoint
        assert ranges[0][0] == 0 and ranges[-1][1] == world * 4 * R  # and contiguous overall
        assert replicas.max_over_ranks(1.5 + rank, dist) == 1.5 + (world - 1)
        rng = np.random.default_rng(10 + rank)
        pk = torch.from_numpy(rng.gamma(2.0, 1.0 + rank, size=(5 + 3 * rank, 7)))
        mean, cov = replicas.merge_mean_cov(pk, dist)
        np.save(os.path.join(out_dir, "pk%d.npy" % rank), pk.numpy())
        np.save(os.path.join(out_dir, "mean%d.npy" % rank), mean.numpy())
        np.save(os.path.join(out_dir, "cov%d.npy" % rank), cov.numpy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path, orc):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    pk = np.concatenate([np.load(tmp_path / ("pk%d.npy" % r)) for r in range(world)])
    ref_mean, ref_cov = orc.mean_cov(pk)
    for r in range(world):
        assert np.allclose(np.load(tmp_path / ("mean%d.npy" % r)), ref_mean, rtol=1e-12)
        assert np.allclose(np.load(tmp_path / ("cov%d.npy" % r)), ref_cov, rtol=1e-10, atol=1e-12)


def test_single_process_and_limits():
    pk = torch.from_numpy(np.random.default_rng(3).normal(size=(9, 4)))
    mean, cov = replicas.merge_mean_cov(pk)
    assert np.allclose(mean.numpy(), pk.numpy().mean(0))
    assert np.allclose(cov.numpy(), np.cov(pk.numpy(), rowvar=False))
    assert replicas.realization_start(3, 8, 2, 64) == (2 * 8 + 3) * 64
    with pytest.raises(ValueError):
        replicas.realization_start(0, 8, 1 << 30, 64)
