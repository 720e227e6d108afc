"""Failure detection through the C ABI, with every failure made on the host side or by a
wait that nothing completes (no fault, trap or unbounded wait on the GPU): a non-finite
Jastrow coefficient makes ratios and E_L non-finite (QMC_ERR_NAN), a stencil copy that is
never issued makes the kernel's bounded wait run out (QMC_ERR_TIMEOUT); in both cases the
crowd works again afterwards."""
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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_nan_coefficient_is_reported_and_recovered(Q, precision):
    wl = wl_mod.pw128()
    W = 8
    c = Q.Crowd.from_workload(wl, precision=precision, n_walkers=W, n_recompute=0)
    R0 = np.ascontiguousarray(wl.positions(n_walkers=W))
    c.qmc_load_positions(R0)
    c.qmc_recompute()
    bad = wl.j2_uu.coefs.copy()
    bad[4] = np.nan  # like-spin pairs at 0.25 < r < 1.25 bohr: about 2 in 5 moves
    c.qmc_load_jastrow(Q.QMC_J2_UU, bad, wl.j2_uu.rc)
    with pytest.raises(Q.QmcError) as ei:
        c.qmc_sweep(1)
    assert ei.value.status == 6
    # moves with a non-finite ratio were rejected; the others went on as usual
    assert np.all(np.isfinite(c.qmc_get_positions()))
    c.qmc_load_jastrow(Q.QMC_J2_UU, wl.j2_uu.coefs, wl.j2_uu.rc)
    e = np.zeros((2, W))
    st = c.qmc_sweep(2, e)
    assert np.all(np.isfinite(e)) and 0.2 < st.n_accept / st.n_moves < 0.95


def test_bounded_wait_times_out_and_the_crowd_recovers(Q):
    """The stencil copy is not issued, so its mbarrier phase never completes: each wait
    gives up after about a second, the sweep returns QMC_ERR_TIMEOUT, no position changes, and after
    the hook is cleared the crowd (rebuilt from its positions) sweeps exactly as a crowd
    that never failed."""
    wl = wl_mod.pw128()
    W = 4
    R0 = np.ascontiguousarray(wl.positions(n_walkers=W))
    ref = Q.Crowd.from_workload(wl, precision="mixed", n_walkers=W, n_recompute=0)
    bad = Q.Crowd.from_workload(wl, precision="mixed", n_walkers=W, n_recompute=0)
    assert bad.kernel_config["stencil_tma"] == 1
    for c in (ref, bad):
        c.qmc_load_positions(R0)
        c.qmc_recompute()
    bad.qmc_test_skip_stencil_copy(True)
    with pytest.raises(Q.QmcError) as ei:
        bad.qmc_sweep(1)
    assert ei.value.status == 5
    assert np.array_equal(bad.qmc_get_positions(), R0)
    bad.qmc_test_skip_stencil_copy(False)
    bad.generation = 0
    out = []
    for c in (ref, bad):
        e = np.zeros((2, W))
        st = c.qmc_sweep(2, e)
        out.append((e, c.qmc_get_positions(), st.n_accept))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    with pytest.raises(Q.QmcError) as ei:
        Q.Crowd.from_workload(wl, precision="mixed", n_walkers=W,
                              staging="ldg").qmc_test_skip_stencil_copy(True)
    assert ei.value.status == 1


def test_non_finite_positions_are_refused(Q):
    """Corrupted inputs: a NaN or infinite coordinate in host memory is refused before
    anything is loaded (INVALID_ARG, the crowd unchanged); one in device memory is
    replaced by 0 and reported as QMC_ERR_NAN by the next synchronising call, and a clean
    reload restores the crowd.  Non-finite ion positions are refused."""
    torch = pytest.importorskip("torch")
    wl = wl_mod.pw128()
    W = 4
    c = Q.Crowd.from_workload(wl, precision="mixed", n_walkers=W, n_recompute=0)
    R0 = np.ascontiguousarray(wl.positions(n_walkers=W))
    c.qmc_load_positions(R0)
    c.qmc_recompute()
    before = c.qmc_get_positions()
    for bad_value in (np.nan, np.inf):
        bad = R0.copy()
        bad[1, 7, 2] = bad_value
        with pytest.raises(Q.QmcError) as ei:
            c.qmc_load_positions(bad)
        assert ei.value.status == 1
        assert np.array_equal(c.qmc_get_positions(), before)
    ions = np.ascontiguousarray(wl.ions.copy())
    ions[0, 0] = np.nan
    with pytest.raises(Q.QmcError) as ei:
        c.qmc_load_ions(ions)
    assert ei.value.status == 1
    bad = R0.copy()
    bad[2, 3, 0] = np.nan
    dev = torch.from_numpy(bad).cuda()
    c.qmc_load_positions(dev)
    with pytest.raises(Q.QmcError) as ei:
        c.qmc_recompute()
    assert ei.value.status == 6
    got = c.qmc_get_positions()
    assert got[2, 3, 0] == 0.0 and np.all(np.isfinite(got))
    c.qmc_load_positions(R0)
    c.qmc_recompute()
    e = np.zeros((1, W))
    st = c.qmc_sweep(1, e)
    assert np.all(np.isfinite(e)) and 0.2 < st.n_accept / st.n_moves < 0.95
