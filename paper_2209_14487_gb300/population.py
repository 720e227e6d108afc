"""A DMC population spread over ranks, one crowd per GPU: the global mixed estimator and
trial-energy feedback, and load balancing by walker exchange.

Walkers are independent (Sec. III), so a rank's crowd needs its neighbours only for the
population-wide sums of a generation and, after branching has made the crowds uneven,
for walkers to even them out.  This module is host bookkeeping over torch.distributed:
it computes nothing of the wavefunction.  A moving walker travels as its positions and
its last local energy; the receiving crowd rebuilds its orbital rows and inverses
(`qmc_dmc_append`), the sending crowd drops it (`qmc_dmc_select`).

The crowd argument needs `W`, `qmc_get_positions()`, `qmc_dmc_select(src)` and
`qmc_dmc_append(R)` (`qmcgb.Crowd` with `dmc=True`).
"""
from __future__ import annotations

import math

import numpy as np


def balance_plan(counts) -> list:
    """Transfers (src, dst, n) that leave rank r with floor(T/R) walkers, plus one for the
    first T mod R ranks (T walkers over R ranks), moving the fewest walkers: ranks above
    their target send to ranks below it, both taken in rank order."""
    R = len(counts)
    T = int(sum(counts))
    if T < R:  # every crowd keeps at least one walker
        return []
    target = [T // R + (1 if r < T % R else 0) for r in range(R)]
    give = [[r, counts[r] - target[r]] for r in range(R) if counts[r] > target[r]]
    take = [[r, target[r] - counts[r]] for r in range(R) if counts[r] < target[r]]
    plan = []
    i = j = 0
    while i < len(give) and j < len(take):
        n = min(give[i][1], take[j][1])
        plan.append((give[i][0], take[j][0], n))
        give[i][1] -= n
        take[j][1] -= n
        if give[i][1] == 0:
            i += 1
        if take[j][1] == 0:
            j += 1
    return plan


def _device(group):
    import torch.distributed as dist
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def global_estimate(w_sum: float, we_sum: float, n_walkers: int, group=None):
    """(E_est, total walkers) over all ranks: E_est = sum w E_L / sum w of the whole
    population, from each rank's sums of one generation."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([w_sum, we_sum, float(n_walkers)], dtype=torch.float64,
                     device=_device(group))
    dist.all_reduce(t, group=group)
    w, we, n = t.tolist()
    return we / w, int(round(n))


def trial_energy(e_est: float, n_total: int, n_target: int, tau: float,
                 feedback: float = 0.1) -> float:
    """E_T = E_est - feedback ln(N / N_target) / tau (population control)."""
    return e_est - feedback * math.log(n_total / n_target) / tau


def exchange(crowd, e_prev, group=None) -> np.ndarray:
    """Evens out the ranks' walker counts (`balance_plan`).  A sending rank gives away its
    last walkers, positions and E_L; a receiving rank appends them in the order of the
    plan (its crowd's capacity must hold ceil(total / ranks) walkers).  Returns this rank's
    E_L array for the new population (host, float64)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = _device(group)
    e_prev = np.ascontiguousarray(e_prev, dtype=np.float64)
    cnt = torch.tensor([crowd.W], dtype=torch.int64, device=dev)
    counts = [torch.zeros_like(cnt) for _ in range(ws)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    plan = balance_plan(counts)
    sends = [(d, n) for s, d, n in plan if s == rank]
    recvs = [(s, n) for s, d, n in plan if d == rank]
    if not sends and not recvs:
        return e_prev
    R = np.asarray(crowd.qmc_get_positions())
    W, N = R.shape[0], R.shape[1]
    per = 3 * N + 1  # one walker: positions, then E_L
    keep = W - sum(n for _, n in sends)
    reqs, inbox = [], []
    for s, n in recvs:
        buf = torch.empty(n * per, dtype=torch.float64, device=dev)
        inbox.append(buf)
        reqs.append(dist.irecv(buf, src=s, group=group))
    off = keep
    outbox = []
    for d, n in sends:
        pay = np.concatenate([R[off:off + n].reshape(n, 3 * N), e_prev[off:off + n, None]],
                             axis=1)
        t = torch.from_numpy(np.ascontiguousarray(pay).reshape(-1)).to(dev)
        outbox.append(t)  # alive until the send completes
        reqs.append(dist.isend(t, dst=d, group=group))
        off += n
    for r in reqs:
        r.wait()
    e_new = e_prev[:keep]
    if sends:
        crowd.qmc_dmc_select(np.arange(keep, dtype=np.int32))
    if recvs:
        got = np.concatenate([b.cpu().numpy().reshape(-1, per) for b in inbox])
        crowd.qmc_dmc_append(np.ascontiguousarray(got[:, :3 * N].reshape(-1, N, 3)))
        e_new = np.concatenate([e_new, got[:, 3 * N]])
    return np.ascontiguousarray(e_new)
