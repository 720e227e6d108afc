"""Several crowds at once (the batched driver's crowds, Sec. III and Alg. 4): crowds on
their own streams driven from concurrent host threads give bit for bit the results of the
same crowds run one after another, including the tensor-core flush (TMEM shared by CTAs
of different crowds on one SM) and a mix of update schemes."""
import dataclasses
import threading

import numpy as np
import pytest

from paper_2209_14487_gb300 import workloads as wl_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14487_gb300 import qmcgb
    return qmcgb


def _run(Q, specs, concurrent, n_gen=3):
    crowds = []
    for i, (wl, precision, update, k) in enumerate(specs):
        c = Q.Crowd.from_workload(wl, precision=precision, update=update, delay_rank=k)
        c.qmc_load_positions(np.ascontiguousarray(wl.positions(crowd_id=i)))
        c.qmc_recompute()
        crowds.append(c)
    out = [np.zeros((n_gen, c.W)) for c in crowds]
    errors = []

    def work(c, o):
        try:
            c.qmc_sweep(n_gen, o)
        except Exception as e:  # re-raised below, in the test's thread
            errors.append(e)

    if concurrent:
        threads = [threading.Thread(target=work, args=(c, o)) for c, o in zip(crowds, out)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    else:
        for c, o in zip(crowds, out):
            work(c, o)
    if errors:
        raise errors[0]
    R = [c.qmc_get_positions() for c in crowds]
    la = [c.qmc_get_logpsi()[0] for c in crowds]
    for c in crowds:
        c.close()
    return out, R, la


def test_concurrent_crowds_match_sequential(Q):
    pw128 = dataclasses.replace(wl_mod.pw128(), n_walkers=48)
    pw512 = dataclasses.replace(wl_mod.pw512(), n_walkers=12)
    specs = [(pw128, "mixed", "sm", 1), (pw128, "mixed", "delayed", 8),
             (pw512, "mixed", "delayed", 16), (pw512, "mixed", "delayed", 16),
             (pw128, "fp64", "sm", 1)]
    seq = _run(Q, specs, concurrent=False)
    con = _run(Q, specs, concurrent=True)
    for a, b in zip(seq[0], con[0]):
        assert np.array_equal(a, b)
    for a, b in zip(seq[1], con[1]):
        assert np.array_equal(a, b)
    for a, b in zip(seq[2], con[2]):
        assert np.array_equal(a, b)


def test_concurrent_fp64_crowds_follow_oracle(Q, oracle_lib):
    """Four FP64 crowds (different starting walkers) swept concurrently from host threads,
    each on its own stream, next to a mixed crowd sharing the GPU: every FP64 crowd's
    trajectory and E_L equal those of an oracle crowd with the same walkers and RNG streams
    (a decision can flip only where u lies within rounding of the acceptance: at most one
    walker per crowd), as in the single-crowd trajectory test."""
    # without drift the trajectories depend on the decisions only, not on the rounding of
    # the drift (which a few hundred dependent moves can amplify past 1e-9)
    wl = dataclasses.replace(wl_mod.pw128(), n_walkers=8, n_recompute=0, drift=False)
    n_gen = 2
    specs = [(wl, "fp64", "sm", 1)] * 4 + [(dataclasses.replace(wl, n_walkers=64), "mixed",
                                            "sm", 1)]
    out, R, _ = _run(Q, specs, concurrent=True, n_gen=n_gen)
    osys = oracle_lib.OracleSystem(wl)
    for i in range(4):
        orc = oracle_lib.OracleCrowd(osys, np.ascontiguousarray(wl.positions(crowd_id=i)))
        e_or, _ = orc.sweep(n_gen)
        d = np.abs(R[i] - orc.positions())
        same = np.all(np.minimum(d, wl.L - d) < 1e-9, axis=(1, 2))
        assert same.sum() >= wl.n_walkers - 1, (i, same)
        rel = np.abs(out[i][:, same] - e_or[:, same]) / np.abs(e_or[:, same])
        assert np.all(rel < 1e-9), (i, rel.max())
