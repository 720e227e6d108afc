"""The mixed path's inverse guard through the C ABI: its probe of A B - I against the same
probe evaluated on the host in FP64 from the crowd's own Slater matrices and inverses, and
its FP64 repair against the crowd's full FP64 recompute."""
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


def probe_signs(n):
    """v_l = -1 where bit 31 of (l + 1) * 0x9E3779B1 (mod 2^32) is set, else +1."""
    h = (np.arange(1, n + 1, dtype=np.uint64) * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)
    return np.where(h >> np.uint64(31), -1.0, 1.0)


def host_probe(c, n):
    """max over spins and k of |(v^T (A B - I))_k| in FP64 on the crowd's FP32 A and B."""
    v = probe_signs(n)
    A = [c.qmc_get_slater_matrix(s) for s in range(2)]
    B = [c.qmc_get_inverse(s) for s in range(2)]
    return np.array([max(np.abs(v @ (A[s][w] @ B[s][w]) - v).max() for s in range(2))
                     for w in range(c.W)])


def test_probe_signs_are_balanced():
    v = probe_signs(1 << 16)
    assert set(np.unique(v)) == {-1.0, 1.0}
    assert abs(v.mean()) < 0.02


@pytest.mark.parametrize("make,update,k,W", [(wl_mod.pw128, "sm", 1, 8),
                                             (wl_mod.pw512, "delayed", 32, 4)])
def test_guard_probe_matches_host(Q, make, update, k, W):
    """With repairs off (a bound no probe reaches) the device's probe after each sweep
    equals the host's FP64 evaluation of the same probe: the double-float sums leave only
    FP32-relative rounding of the result."""
    wl = make()
    c = Q.Crowd.from_workload(wl, precision="mixed", update=update, delay_rank=k, n_walkers=W,
                              n_recompute=0, guard_tol=1e30)
    c.qmc_load_positions(np.ascontiguousarray(wl.positions(n_walkers=W)))
    c.qmc_recompute()
    for _ in range(2):
        st = c.qmc_sweep(1)
        assert st.n_repair == 0
        g, n_rep = c.qmc_get_guard()
        assert n_rep == 0
        ref = host_probe(c, wl.n_up)
        assert np.all(ref > 0)
        assert np.allclose(g, ref, rtol=1e-5, atol=1e-9), (g, ref)


@pytest.mark.parametrize("update,k", [("delayed", 8), ("sm", 1)])
def test_guard_repair_equals_fp64_recompute(Q, update, k):
    """A bound below every probe repairs every walker after every sweep: each inverse is
    then the FP64 inverse of the crowd's own (FP32) Slater matrix rounded to FP32, and
    log|Psi| and E_L equal those of a full FP64 recompute at the same positions."""
    wl = wl_mod.pw128()
    W = 8
    n = wl.n_up
    c = Q.Crowd.from_workload(wl, precision="mixed", update=update, delay_rank=k, n_walkers=W,
                              n_recompute=0, guard_tol=1e-30)
    c.qmc_load_positions(np.ascontiguousarray(wl.positions(n_walkers=W)))
    c.qmc_recompute()
    e = np.zeros((2, W))
    st = c.qmc_sweep(2, e)
    assert st.n_repair == 2 * W
    assert c.qmc_get_guard()[1] == 2 * W
    for s in range(2):
        A = c.qmc_get_slater_matrix(s)
        B = c.qmc_get_inverse(s)
        for w in range(W):
            ref = np.linalg.inv(A[w])
            assert np.allclose(B[w], ref, rtol=2.0 ** -22, atol=2.0 ** -22 * np.abs(ref).max())
    la1, sg1 = c.qmc_get_logpsi()
    c.qmc_recompute()
    la2, sg2 = c.qmc_get_logpsi()
    e2 = np.zeros(W)
    c.qmc_local_energy_batch(e2)
    assert np.array_equal(sg1, sg2)
    assert np.allclose(la1, la2, rtol=1e-6, atol=1e-6), np.abs(la1 - la2).max()
    assert np.allclose(e[-1], e2, rtol=1e-4, atol=1e-4), np.abs(e[-1] - e2).max()


def test_guard_settings(Q):
    wl = wl_mod.pw16()
    off = Q.Crowd.from_workload(wl, precision="mixed", guard_tol=-1.0)
    with pytest.raises(Q.QmcError) as ei:
        off.qmc_get_guard()
    assert ei.value.status == 7
    f64 = Q.Crowd.from_workload(wl, precision="fp64")
    with pytest.raises(Q.QmcError) as ei:
        f64.qmc_get_guard()
    assert ei.value.status == 7
    with pytest.raises(Q.QmcError) as ei:
        Q.Crowd.from_workload(wl, precision="mixed", guard_tol=float("nan"))
    assert ei.value.status == 1
    on = Q.Crowd.from_workload(wl, precision="mixed")
    on.qmc_load_positions(np.ascontiguousarray(wl.positions()))
    st = on.qmc_sweep(3)
    g, n_rep = on.qmc_get_guard()
    assert n_rep == st.n_repair == 0 and np.all(g < 1e-3) and np.all(g >= 0)
