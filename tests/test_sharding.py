"""Multi-process (gloo, world size 2, CPU) checks of the walker-sharded VMC
step: the gathered clipping weights, the all-reduced gradient and the global
energy mean and variance (merged from per-rank centred moments) equal the single-process results on the whole batch."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2307_14123_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, B, P, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(0)
    e_all = rng.standard_cauchy(B) * 2 - 30
    g_all = rng.normal(size=(B, P))
    off, cnt = sharding.shard(B, rank, world)
    e_loc = torch.tensor(e_all[off:off + cnt])
    w = sharding.global_loss_weights(e_loc, lambda e: torch.tensor(oracle.clipped_loss_weights(e.numpy(), 5.0)[0]))
    g = torch.tensor(w.numpy() @ g_all[off:off + cnt])
    sharding.allreduce_gradient(g)
    mean, var = sharding.global_energy(e_loc)
    # an offset of 1e9 Ha with a spread of a few Ha: the centred merge keeps the variance
    mean_off, var_off = sharding.global_energy(e_loc + 1e9)
    q.put((rank, off, cnt, w.numpy(), g.numpy(), float(mean), float(var), float(mean_off), float(var_off)))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_step_equals_unsharded():
    B, P, world = 1001, 7, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, B, P, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(0)
    e_all = rng.standard_cauchy(B) * 2 - 30
    g_all = rng.normal(size=(B, P))
    w_ref = oracle.clipped_loss_weights(e_all, 5.0)[0]
    assert sum(r[2] for r in res) == B and res[0][1] == 0 and res[1][1] == res[0][2]
    np.testing.assert_allclose(np.concatenate([r[3] for r in res]), w_ref, rtol=1e-13, atol=1e-16)
    for r in res:
        np.testing.assert_allclose(r[4], w_ref @ g_all, rtol=1e-12, atol=1e-14)
        assert abs(r[5] - e_all.mean()) < 1e-10 * max(1, abs(e_all.mean()))
        assert abs(r[6] - e_all.var()) < 1e-8 * e_all.var()
        assert abs(r[7] - (e_all.mean() + 1e9)) < 1e-6
        assert abs(r[8] - e_all.var()) < 1e-6 * e_all.var()


def test_shard_covers_every_walker_once():
    for B in (1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                off, cnt = sharding.shard(B, r, world)
                seen += list(range(off, off + cnt))
            assert seen == list(range(B))
