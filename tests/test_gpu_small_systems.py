"""The smallest systems against the oracle: one and two electrons per spin (N = 2, 4) and a
tiny system with ions (N = 8), in both precisions and both update schemes.  These are
also the cases the bounds-checked build runs (QMCGB_CHECK=1 loads libqmcgb_check.so, see
test_gpu_checked.py): there every device index check must stay silent, and a planted
out-of-range spline cell must be caught before any load."""
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


def _system(n_el):
    if n_el == 8:
        return wl_mod.tiny(n_el=8, n_walkers=5)
    return wl_mod.make_workload(f"e{n_el}", n_el=n_el, n_orb=n_el // 2, grid=6, n_walkers=5,
                                n_gen=1, n_ions=2, L=2.0 + 0.5 * n_el, j1_knots=5,
                                j2_knots=6, tau=0.3)


CASES = [(2, "fp64", "sm", 1), (4, "fp64", "sm", 1), (4, "fp64", "delayed", 2),
         (4, "mixed", "sm", 1), (8, "fp64", "delayed", 3), (8, "mixed", "delayed", 2),
         (8, "mixed", "sm", 1)]


def test_loaded_build_is_the_requested_one(Q):
    assert Q.build_flags() == (Q.QMC_BUILD_CHECKED if Q.CHECKED else 0)


@pytest.mark.parametrize("n_el,precision,update,k", CASES)
def test_small_system_against_oracle(Q, oracle_lib, n_el, precision, update, k):
    """Three generations on the internal RNG.  FP64: positions and E_L follow the oracle's
    trajectory to 1e-9 (one walker may leave it on a decision within rounding of u).
    Mixed: log|Psi| and E_L at the GPU's positions equal the oracle's to 1e-4 and 1e-3."""
    wl = _system(n_el)
    W = wl.n_walkers
    R = np.ascontiguousarray(wl.positions(n_walkers=W))
    gpu = Q.Crowd.from_workload(wl, precision=precision, update=update, delay_rank=k,
                                n_walkers=W)
    gpu.qmc_load_positions(R)
    gpu.qmc_recompute()
    osys = oracle_lib.OracleSystem(wl)
    n_gen = 3
    e = np.zeros((n_gen, W))
    st = gpu.qmc_sweep(n_gen, e)
    assert st.n_moves == n_gen * W * n_el
    Rg = gpu.qmc_get_positions()
    if precision == "fp64":
        orc = oracle_lib.OracleCrowd(osys, R)
        e_or, _ = orc.sweep(n_gen)
        same = np.all(np.abs(Rg - orc.positions()) < 1e-9, axis=(1, 2))
        assert same.sum() >= W - 1, same
        assert np.allclose(e[:, same], e_or[:, same], rtol=1e-9, atol=1e-9)
    else:
        la, sg = gpu.qmc_get_logpsi()
        for w in range(W):
            ref, rsg = osys.logpsi(Rg[w])
            assert abs(la[w] - ref) < 1e-4 * max(1.0, abs(ref)), (w, la[w], ref)
            assert sg[w] == rsg
            e_ref = osys.local_energy(Rg[w])[0]
            assert abs(e[-1, w] - e_ref) < 1e-3 * max(1.0, abs(e_ref)), (w, e[-1, w], e_ref)
    assert gpu.qmc_check_report() == (0, 0)


def test_planted_bad_cell_is_caught(Q):
    """Checked build only: electron 0's proposals get spline cell G + 5 (outside the
    table); the cell check records it and replaces it by cell 0 before any load, the sweep
    returns QMC_ERR_BOUNDS, and once the hook is cleared the crowd (rebuilt from its
    stored positions) sweeps cleanly.  The normal build refuses the hook (UNSUPPORTED)."""
    wl = _system(8)
    for precision in ("fp64", "mixed"):
        c = Q.Crowd.from_workload(wl, precision=precision)
        c.qmc_load_positions(np.ascontiguousarray(wl.positions()))
        c.qmc_recompute()
        if not Q.CHECKED:
            with pytest.raises(Q.QmcError) as ei:
                c.qmc_test_plant_bad_cell(True)
            assert ei.value.status == Q.QMC_ERR_UNSUPPORTED
            continue
        c.qmc_test_plant_bad_cell(True)
        with pytest.raises(Q.QmcError) as ei:
            c.qmc_sweep(1)
        assert ei.value.status == Q.QMC_ERR_BOUNDS
        site, value = c.qmc_check_report()
        assert site == 3 and value == wl.grid + 5, (site, value)  # x dimension (0 << 32)
        assert c.qmc_check_report() == (0, 0)  # the report clears
        assert np.all(np.isfinite(c.qmc_get_positions()))
        c.qmc_test_plant_bad_cell(False)
        e = np.zeros((2, c.W))
        st = c.qmc_sweep(2, e)
        assert np.all(np.isfinite(e)) and 0.2 < st.n_accept / st.n_moves < 0.98
        assert c.qmc_check_report() == (0, 0)
