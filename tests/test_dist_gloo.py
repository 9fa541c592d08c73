"""Data-parallel host logic on CPU: two gloo ranks, each with its own shard of a 4f batch.

The per-rank gradients come from the oracle (this checks the sharding and the reduction,
not the kernels): the mean of the ranks' pupil-phase gradients must equal the gradient of
the mean loss over the whole batch.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
import synthetic as S
from paper_2411_18591_gb300 import dist as D

N, COMPS, NLAM, OBJECTS = 16, 1, 2, 4
D_M, F_M, LENS_R, PUPIL_R = 20e-6, 0.05, 150e-6, 100e-6


def _problem(first, count):
    obj = S.cfg4_objects(count, COMPS, N, first=first).reshape(-1, N, N)
    fields = np.repeat(obj, NLAM, axis=0).astype(np.complex128)  # (object, component, wavelength)
    lams = np.tile(np.linspace(450e-9, 700e-9, NLAM), count * COMPS)
    target = S.cfg4_target(count, N, first=first)
    return fields, lams, target


def _phase():
    return S.uniform(S.sub_seed(S.BASE_SEED, 77), (N, N), -np.pi, np.pi)


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = D.shard(OBJECTS, rank, world)
        fields, lams, target = _problem(mine.start, len(mine))
        _, g, _ = O.fourf_loss_and_grad(fields, lams, D_M, F_M, LENS_R, PUPIL_R, _phase(), COMPS * NLAM, target)
        grad = torch.from_numpy(np.ascontiguousarray(g))
        D.average_gradient(grad)
        if rank == 0:
            np.save(out_path, grad.numpy())
    finally:
        torch.distributed.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_every_item_once():
    for n in (0, 1, 5, 16, 17, 384):
        for world in (1, 2, 3, 8):
            parts = [D.shard(n, r, world) for r in range(world)]
            assert [i for p in parts for i in p] == list(range(n))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def test_two_rank_mean_gradient_equals_full_batch(tmp_path):
    out = tmp_path / "g.npy"
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    fields, lams, target = _problem(0, OBJECTS)
    _, g_full, _ = O.fourf_loss_and_grad(fields, lams, D_M, F_M, LENS_R, PUPIL_R, _phase(), COMPS * NLAM, target)
    g_ranks = np.load(out)
    assert np.abs(g_full).max() > 0
    np.testing.assert_allclose(g_ranks, g_full, rtol=1e-12, atol=1e-12 * np.abs(g_full).max())
