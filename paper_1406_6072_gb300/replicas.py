"""Replicas across processes (one GPU each): the path shards by realization.

Realizations are independent and drawn from counter-based streams, so rank r
of W draws realizations [(s W + r) R, (s W + r + 1) R) at step s: disjoint
for every (rank, step), identical on any device.  The only exchange is after
the fact: the max of the ranks' step times, and the mean and covariance of
the binned power spectra over all ranks' fields (each rank's count, mean and
centred second moment, combined with the pairwise update of Chan, Golub and
LeVeque, so no rank needs another's spectra).  Works with any
torch.distributed backend (gloo on CPU in the tests).
"""
from __future__ import annotations

import torch


def realization_start(rank: int, world: int, step: int, R: int) -> int:
    """First realization of rank `rank` at step `step` (R per rank and step)."""
    r0 = (step * world + rank) * R
    if r0 + R > 1 << 32:
        raise ValueError("realization index exceeds 32 bits")
    return r0


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest `value` over the ranks (the step time of the slowest rank)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def merge_mean_cov(pk: torch.Tensor, dist=None):
    """Mean [nb] and unbiased covariance [nb, nb] over the fields of all ranks.
    pk: this rank's spectra [F, nb] (binary64, any device; moved to the CPU
    for the exchange).  Every rank returns the same result."""
    x = pk.detach().to("cpu", torch.float64)
    n = torch.tensor(float(x.shape[0]), dtype=torch.float64)
    mean = x.mean(0) if x.shape[0] else torch.zeros(x.shape[1], dtype=torch.float64)
    d = x - mean
    m2 = d.T @ d
    if dist is None or dist.get_world_size() == 1:
        parts = [(n, mean, m2)]
    else:
        world = dist.get_world_size()
        ns = [torch.zeros_like(n) for _ in range(world)]
        means = [torch.zeros_like(mean) for _ in range(world)]
        m2s = [torch.zeros_like(m2) for _ in range(world)]
        dist.all_gather(ns, n)
        dist.all_gather(means, mean)
        dist.all_gather(m2s, m2)
        parts = list(zip(ns, means, m2s))
    # combine in rank order: n = na + nb, delta = mb - ma,
    # mean = ma + delta nb / n, M2 = M2a + M2b + delta delta^T na nb / n
    na, ma, qa = parts[0]
    for nb_, mb, qb in parts[1:]:
        tot = na + nb_
        if tot == 0:
            continue
        delta = mb - ma
        ma = ma + delta * (nb_ / tot)
        qa = qa + qb + torch.outer(delta, delta) * (na * nb_ / tot)
        na = tot
    cov = qa / (na - 1) if na > 1 else torch.zeros_like(qa)
    return ma, cov
