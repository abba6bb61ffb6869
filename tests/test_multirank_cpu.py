"""The multi-rank split on CPU ranks (gloo, world size 2).

The GPU kernels are not involved: each rank computes its partial mode-1 Gram
matrix with the oracle, the partials are summed by the same all-reduce the
multi-GPU training side uses, and the shards of the test pass are checked to
cover every matrix exactly once.  The refiner's data-parallel SGD is run
with the oracle's gradient on each rank's half of every batch and must give
the same steps as one process on the whole batches.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2209_14637_gb300.dist import (allreduce_gram, allreduce_mean, data_parallel_sgd,
                                         shard_range)


def test_shard_ranges_partition():
    for count in (0, 1, 7, 500, 513):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                a, b = shard_range(count, world, r)
                assert 0 <= a <= b <= count
                seen.extend(range(a, b))
            assert seen == list(range(count))
            sizes = [shard_range(count, world, r)[1] - shard_range(count, world, r)[0]
                     for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, As, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    a, b = shard_range(len(As), world, rank)
    G = torch.tensor(oracle.gram_mode1(As[a:b]) if b > a else
                     np.zeros((As[0].shape[0],) * 2))
    allreduce_gram(G)
    S, _ = oracle.leading_eigvecs(G.numpy(), 3)
    out[rank] = (G.numpy(), S)
    dist.barrier()
    dist.destroy_process_group()


def test_partial_grams_sum_to_the_full_gram():
    rng = np.random.default_rng(0)
    As = [rng.standard_normal((12, 9)) for _ in range(7)]
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), As, out), nprocs=world, join=True)
    import oracle
    G = oracle.gram_mode1(As)
    S, _ = oracle.leading_eigvecs(G, 3)
    for r in range(world):
        Gr, Sr = out[r]
        np.testing.assert_allclose(Gr, G, rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(Sr, S, atol=1e-12)


def test_allreduce_rejects_low_precision():
    with pytest.raises(ValueError):
        allreduce_gram(torch.zeros(2, 2, dtype=torch.float32))


def _batches(step, As, lo, hi):
    """Step `step` uses matrices 4 step .. 4 step + 3 (cyclic); a rank takes
    [lo, hi) of those four."""
    idx = [(4 * step + i) % len(As) for i in range(4)]
    return [As[i] for i in idx[lo:hi]]


def _sgd_worker(rank, world, port, As, S0, r, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    lo, hi = shard_range(4, world, rank)

    def grad(S, batch):
        return torch.tensor(oracle.ivy_grad(S.numpy(), batch, r))

    dS = data_parallel_sgd(grad, torch.tensor(S0), lambda t: _batches(t, As, lo, hi),
                           steps=3, lr=0.05)
    out[rank] = dS.numpy()
    dist.barrier()
    dist.destroy_process_group()


def test_data_parallel_refiner_steps_match_one_process():
    import oracle
    rng = np.random.default_rng(1)
    As = [rng.standard_normal((10, 8)) @ np.diag(np.linspace(3, 0.2, 8)) for _ in range(8)]
    S0 = np.linalg.qr(rng.standard_normal((10, 4)))[0].T
    r = 2
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_sgd_worker, args=(world, _free_port(), As, S0, r, out), nprocs=world, join=True)
    dS = np.zeros_like(S0)
    for step in range(3):
        dS -= 0.05 * oracle.ivy_grad(S0 + dS, _batches(step, As, 0, 4), r)
    assert np.abs(dS).max() > 1e-6  # the steps move S
    for rk in range(world):
        np.testing.assert_allclose(out[rk], dS, rtol=1e-11, atol=1e-13)


def test_allreduce_mean_without_a_group_is_the_identity():
    t = torch.tensor([1.0, 2.0])
    assert torch.equal(allreduce_mean(t), torch.tensor([1.0, 2.0]))
    with pytest.raises(ValueError):
        allreduce_mean(torch.tensor([1, 2]))
