"""Batches of crowds of different sizes (64, 192 and 384 electrons) swept by one launch
per generation: the result equals each crowd's own qmc_sweep, and every system agrees
with the FP64 oracle's recompute at the walkers' positions."""
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


WALKERS = (6, 4, 3)  # per system: the batch covers three crowds of different sizes


def _crowds(Q, precision, update="sm", k=1, n_recompute=(0, 2, 0), nt=128):
    out = []
    for make, W, nrc in zip(wl_mod.MIXED_BATCH, WALKERS, n_recompute):
        wl = make()
        c = Q.Crowd.from_workload(wl, precision=precision, update=update, delay_rank=k,
                                  n_walkers=W, n_recompute=nrc, cta_threads=nt)
        c.qmc_load_positions(np.ascontiguousarray(wl.positions(n_walkers=W)))
        c.qmc_recompute()
        out.append((wl, c))
    return out


@pytest.mark.parametrize("precision,update,k", [("mixed", "sm", 1), ("fp64", "sm", 1),
                                                ("mixed", "delayed", 4)])
def test_batch_equals_separate_sweeps(Q, precision, update, k):
    a = _crowds(Q, precision, update, k)
    b = _crowds(Q, precision, update, k)
    batch = Q.Batch([c for _, c in a])
    n_gen = 3  # the 192-electron crowd recomputes after its second generation
    e_batch, st_batch = batch.qmc_batch_sweep(n_gen)
    assert batch.launch_count > 0
    for (wl, ca), (_, cb), eb, sb in zip(a, b, e_batch, st_batch):
        e_sep = np.zeros((n_gen, ca.W))
        s_sep = cb.qmc_sweep(n_gen, e_sep)
        assert ca.generation == cb.generation == n_gen
        assert np.array_equal(ca.qmc_get_positions(), cb.qmc_get_positions()), wl.name
        assert np.allclose(eb, e_sep, rtol=1e-12, atol=0), wl.name
        assert sb.n_accept == s_sep.n_accept
        assert sb.n_moves == s_sep.n_moves == n_gen * ca.W * wl.n_el
        la, _ = ca.qmc_get_logpsi()
        lb, _ = cb.qmc_get_logpsi()
        assert np.allclose(la, lb, rtol=1e-12, atol=1e-12)
    batch.close()


def test_batch_systems_match_oracle(Q, oracle_lib):
    """Per-system error of the mixed batch against the FP64 oracle's full recompute at the
    GPU's positions after the sweeps: log|Psi| and E_L."""
    crowds = _crowds(Q, "mixed")
    batch = Q.Batch([c for _, c in crowds])
    e, st = batch.qmc_batch_sweep(2)
    for (wl, c), el, s in zip(crowds, e, st):
        assert 0.2 < s.n_accept / s.n_moves < 0.95, wl.name
        R = c.qmc_get_positions()
        la, sg = c.qmc_get_logpsi()
        osys = oracle_lib.OracleSystem(wl)
        for w in range(min(2, c.W)):
            ref, rsg = osys.logpsi(R[w])
            assert abs(la[w] - ref) < 1e-4 * max(1.0, abs(ref)), (wl.name, la[w], ref)
            assert sg[w] == rsg
            e_ref = osys.local_energy(R[w])[0]
            assert abs(el[-1, w] - e_ref) < 1e-3 * max(1.0, abs(e_ref)), (wl.name, el[-1, w], e_ref)
    batch.close()


def test_batch_rejects_mismatched_crowds(Q):
    wl = wl_mod.tiny()
    a = Q.Crowd.from_workload(wl, precision="mixed", cta_threads=128)
    b = Q.Crowd.from_workload(wl, precision="fp64", cta_threads=128)
    c = Q.Crowd.from_workload(wl, precision="mixed", cta_threads=256)
    for pair in ([a, b], [a, c], [a, a]):
        with pytest.raises(Q.QmcError):
            Q.Batch(pair)
