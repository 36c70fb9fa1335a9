"""Walker sharding across GPUs, one process per GPU.

Walkers are independent Markov chains (Sec. 5), so the hot path shards by
walkers: each rank holds its own walkers and runs ansatz_eval, local_energy,
mcmc_step and grad_logpsi on them without any exchange.  A distributed VMC
step has two exchange steps, both on the host side of the library:

* the clipping window of Sec. 4.4 needs the median and the mean absolute
  deviation of all walkers' local energies: the local energies are
  all-gathered (B floats), every rank computes the weights of the whole batch
  with the same kernel and keeps its own slice, so the result equals the
  single-process one exactly;
* the gradient estimator of Eq. (30) sums over all walkers: the weighted
  gradients of the ranks are all-reduced (P values).

Throughput runs (bench.py) need neither and report weak scaling.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(B_global: int, rank: int, world: int):
    """(offset, count) of this rank's walkers; counts differ by at most one."""
    base, extra = divmod(int(B_global), int(world))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def gather_local_energies(e_local: torch.Tensor, group=None) -> torch.Tensor:
    """All local energies of all ranks, in rank order."""
    world = dist.get_world_size(group)
    n = torch.tensor([e_local.numel()], device=e_local.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    m = int(max(int(x.item()) for x in sizes))
    buf = torch.zeros(m, dtype=e_local.dtype, device=e_local.device)
    buf[: e_local.numel()] = e_local
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[: int(k.item())] for p, k in zip(parts, sizes)])


def global_loss_weights(e_local: torch.Tensor, weights_fn, group=None):
    """This rank's slice of the clipped gradient weights of the whole batch.

    ``weights_fn(e_all) -> weights_all`` computes the weights of a full batch
    (``Ansatz.vmc_loss_weights`` on a GPU).
    """
    e_all = gather_local_energies(e_local, group)
    w_all = weights_fn(e_all)
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    off, cnt = shard(e_all.numel(), rank, world)
    # ranks hold shard() slices of the batch
    return w_all[off:off + cnt]


def allreduce_gradient(g: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the ranks' weighted gradients (in place)."""
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g


def global_energy(e_local: torch.Tensor, group=None):
    """Mean and variance of the local energy over all ranks' walkers, from each rank's local
    energies.  Each rank forms its count, mean and centred sum of squares M2 = sum (E - mean)^2
    in FP64; the ranks' triples are all-gathered and merged in rank order by the pairwise update
    of Chan, Golub and LeVeque (1979): n = n_a + n_b, d = mean_b - mean_a, mean = mean_a + d n_b / n,
    M2 = M2_a + M2_b + d^2 n_a n_b / n.  No step subtracts two large moments, so the variance keeps
    its relative accuracy when |mean| is much larger than the spread (E[x^2] - mean^2 would not).
    Non-finite energies are excluded."""
    e = e_local.detach().double().reshape(-1)
    e = e[torch.isfinite(e)]
    n = float(e.numel())
    mu = float(e.mean()) if n else 0.0
    m2 = float(((e - mu) ** 2).sum()) if n else 0.0
    mine = torch.tensor([n, mu, m2], dtype=torch.float64, device=e_local.device)
    world = dist.get_world_size(group)
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    n_a, mean_a, m2_a = 0.0, 0.0, 0.0
    for p in parts:
        n_b, mean_b, m2_b = (float(x) for x in p)
        if n_b == 0:
            continue
        tot = n_a + n_b
        d = mean_b - mean_a
        mean_a = mean_a + d * n_b / tot
        m2_a = m2_a + m2_b + d * d * n_a * n_b / tot
        n_a = tot
    return mean_a, (m2_a / n_a if n_a else float("nan"))
