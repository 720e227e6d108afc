"""The benchmark configurations at their full sizes and in the launch configurations the
bench times (the autotuner's picks on GB300): sampled walkers after whole generations
against the FP64 oracle's recompute at the GPU's positions.  pw512: 1024 walkers, delayed
k = 32, 256 threads; the mixed-size batch: 512/256/128 walkers in one launch per
generation; dmc1536: 512 walkers, delayed k = 32, 128 threads, a DMC generation with
branching."""
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


def test_pw512_bench_configuration(Q, oracle_lib):
    wl = wl_mod.pw512()
    gpu = Q.Crowd.from_workload(wl, precision="mixed", update="delayed", delay_rank=32,
                                cta_threads=256)
    cfg = gpu.kernel_config
    assert cfg["cta_threads"] == 256 and cfg["tc_flush"] == 1
    gpu.qmc_load_positions(np.ascontiguousarray(wl.positions()))
    gpu.qmc_recompute()
    e = np.zeros((2, wl.n_walkers))
    st = gpu.qmc_sweep(2, e)
    assert 0.5 < st.n_accept / st.n_moves < 0.95
    R = gpu.qmc_get_positions()
    la, sg = gpu.qmc_get_logpsi()
    osys = oracle_lib.OracleSystem(wl)
    for w in [0, 511, 1023]:
        ref, rs = osys.logpsi(R[w])
        assert abs(la[w] - ref) < 1e-4 * max(1.0, abs(ref)) and sg[w] == rs
        e_ref = osys.local_energy(R[w])[0]
        assert abs(e[-1, w] - e_ref) < 1e-3 * max(1.0, abs(e_ref)), (w, e[-1, w], e_ref)


def test_mixed_size_batch_bench_configuration(Q, oracle_lib):
    crowds = []
    for make in wl_mod.MIXED_BATCH:
        wl = make()
        c = Q.Crowd.from_workload(wl, precision="mixed", cta_threads=128)
        c.qmc_load_positions(np.ascontiguousarray(wl.positions()))
        c.qmc_recompute()
        crowds.append((wl, c))
    batch = Q.Batch([c for _, c in crowds])
    e, st = batch.qmc_batch_sweep(2)
    for (wl, c), el, s in zip(crowds, e, st):
        assert el.shape == (2, wl.n_walkers)
        assert 0.2 < s.n_accept / s.n_moves < 0.95
        R = c.qmc_get_positions()
        la, _ = c.qmc_get_logpsi()
        osys = oracle_lib.OracleSystem(wl)
        for w in [0, wl.n_walkers - 1]:
            ref, _ = osys.logpsi(R[w])
            assert abs(la[w] - ref) < 1e-4 * max(1.0, abs(ref)), (wl.name, w)
            e_ref = osys.local_energy(R[w])[0]
            assert abs(el[-1, w] - e_ref) < 1e-3 * max(1.0, abs(e_ref)), (wl.name, w)
    batch.close()


def test_dmc1536_bench_configuration(Q, oracle_lib):
    """A DMC generation and its branching at full size; E_L to 1e-3 and log|Psi| to 1e-4
    for every sampled walker of the new population (the inverse guard recomputes in FP64
    any inverse that drifted during the generation, before its E_L)."""
    wl = wl_mod.dmc1536()
    gpu = Q.Crowd.from_workload(wl, precision="mixed", update="delayed", delay_rank=32,
                                cta_threads=128, dmc=True)
    cfg = gpu.kernel_config
    assert cfg["tc_flush"] == 1 and cfg["cta_threads"] == 128
    gpu.qmc_load_positions(np.ascontiguousarray(wl.positions()))
    gpu.qmc_recompute()
    e_prev = np.zeros(wl.n_walkers)
    gpu.qmc_local_energy_batch(e_prev)
    e_new = np.zeros((1, wl.n_walkers))
    sw = gpu.qmc_sweep(1, e_new)
    g, n_rep = gpu.qmc_get_guard()
    assert sw.n_repair == n_rep == int(np.sum(~(g <= 0.1)))
    st, e_next = gpu.qmc_dmc_branch(e_prev, e_new[0], float(e_prev.mean()))
    assert st.n_before == wl.n_walkers and 0 < st.n_after <= wl.n_walkers
    assert gpu.walker_count == st.n_after == len(e_next)
    assert np.all(np.isfinite(e_next))
    # keep three walkers of the new population (their state copied as is) and check them
    sample = [0, st.n_after // 2, st.n_after - 1]
    gpu.qmc_dmc_select(sample)
    R = gpu.qmc_get_positions()
    la, _ = gpu.qmc_get_logpsi()
    osys = oracle_lib.OracleSystem(wl)
    for w in range(3):
        ref, _ = osys.logpsi(R[w])
        assert abs(la[w] - ref) < 1e-4 * max(1.0, abs(ref)), (w, la[w], ref)
        e_ref = osys.local_energy(R[w])[0]
        e_gpu = e_next[sample[w]]
        assert abs(e_gpu - e_ref) < 1e-3 * abs(e_ref), (w, e_gpu, e_ref)
