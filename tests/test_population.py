"""Walker exchange between ranks (one crowd per GPU) over CPU ranks (gloo), with crowds
stood in for by host arrays that keep the same population calls: balancing conserves
every walker and its local energy, evens the counts, and the global estimator sums the
ranks' weights."""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2209_14487_gb300 import population


def test_balance_plan():
    assert population.balance_plan([5, 5, 5]) == []
    assert population.balance_plan([9, 2, 7]) == [(0, 1, 3), (2, 1, 1)]
    plan = population.balance_plan([0, 13, 1, 6])
    counts = [0, 13, 1, 6]
    for s, d, n in plan:
        assert n > 0 and counts[s] - n >= 0
        counts[s] -= n
        counts[d] += n
    assert counts == [5, 5, 5, 5]
    assert population.balance_plan([1, 0, 0]) == []  # fewer walkers than ranks


def test_trial_energy_feedback():
    assert population.trial_energy(-2.0, 100, 100, 0.01) == -2.0
    assert population.trial_energy(-2.0, 200, 100, 0.01) == pytest.approx(
        -2.0 - 0.1 * math.log(2.0) / 0.01)


class _HostCrowd:
    """The population calls of a DMC crowd on host arrays."""

    def __init__(self, R):
        self.R = np.array(R)
        self.W = len(self.R)

    def qmc_get_positions(self):
        return self.R.copy()

    def qmc_dmc_select(self, src):
        self.R = self.R[np.asarray(src)]
        self.W = len(self.R)

    def qmc_dmc_append(self, R):
        self.R = np.concatenate([self.R, R])
        self.W = len(self.R)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


COUNTS = [9, 2, 7]
N_EL = 4


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    W = COUNTS[rank]
    ids = 1000.0 * rank + np.arange(W)
    R = np.zeros((W, N_EL, 3))
    R[:, :, 0] = ids[:, None]
    R[:, :, 1] = np.arange(N_EL)[None, :]
    crowd = _HostCrowd(R)
    e = population.exchange(crowd, ids + 0.5)
    est, n_total = population.global_estimate(float(rank + 1), 2.0 * (rank + 1), W)
    q.put((rank, crowd.R.tolist(), e.tolist(), est, n_total))
    dist.destroy_process_group()


def test_exchange_over_three_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ws = len(COUNTS)
    ps = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    seen = []
    for rank, R, e, est, n_total in out:
        R, e = np.array(R), np.array(e)
        assert len(R) == 6  # 18 walkers over 3 ranks
        assert np.array_equal(R[:, :, 1], np.tile(np.arange(N_EL), (6, 1)))
        assert np.all(R[:, :, 0] == R[:, :1, 0])  # each walker arrived whole
        assert np.array_equal(e, R[:, 0, 0] + 0.5)  # with its own E_L
        assert est == 2.0 and n_total == sum(COUNTS)
        seen.extend(R[:, 0, 0].tolist())
    expect = [1000.0 * r + w for r, c in enumerate(COUNTS) for w in range(c)]
    assert sorted(seen) == sorted(expect)
    # the ranks that gave walkers kept their first ones, in order
    assert out[0][1][0][0][0] == 0.0 and out[2][1][0][0][0] == 2000.0
