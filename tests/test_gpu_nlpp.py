"""The nonlocal pseudopotential term of E_L on the GPU (a kernel of its own after every
E_L launch) against the FP64 oracle: FP64 to 1e-10 on fresh E_L and through sweeps, the
mixed path to the mixed E_L tolerance at the bench workload's geometry; argument checks
and the batch refusal."""
import numpy as np
import pytest

from paper_2209_14487_gb300 import workloads as wl_mod

pytestmark = pytest.mark.gpu

AMPS, WIDTHS = (1.2, -0.8, 0.5), (0.7, 0.9, 0.8)


@pytest.fixture(scope="module")
def Q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14487_gb300 import qmcgb
    return qmcgb


def _ions26():
    # 26 electrons (13 per spin: ragged orbital tiles), 5 ions, J1 + J2 + potential
    return wl_mod.make_workload("nl26", n_el=26, n_orb=15, grid=14, n_walkers=7, n_gen=3,
                                n_ions=5, L=5.3, tau=0.4, j1_knots=7, j2_knots=9)


@pytest.mark.parametrize("update,k", [("sm", 1), ("delayed", 3)])
def test_nlpp_fp64_matches_oracle(Q, oracle_lib, update, k):
    wl = _ions26()
    rc = 2.0
    R = np.ascontiguousarray(wl.positions())
    gpu = Q.Crowd.from_workload(wl, precision="fp64", update=update, delay_rank=k)
    gpu.qmc_load_nlpp(AMPS, WIDTHS, rc)
    gpu.qmc_load_positions(R)
    gpu.qmc_recompute()
    e = np.zeros(wl.n_walkers)
    gpu.qmc_local_energy_batch(e)
    osys = oracle_lib.OracleSystem(wl, nlpp=(AMPS, WIDTHS, rc),
                                   update=1 if update == "delayed" else 0, delay_rank=k)
    ref = np.array([osys.local_energy(R[w])[0] for w in range(wl.n_walkers)])
    nl = np.array([osys.nlpp(R[w]) for w in range(wl.n_walkers)])
    assert np.count_nonzero(np.abs(nl) > 1e-3) >= 3
    assert np.allclose(e, ref, rtol=1e-10, atol=1e-10)
    # through sweeps: every generation's E_L against the oracle crowd's
    e2 = np.zeros((2, wl.n_walkers))
    gpu.qmc_sweep(2, e2)
    orc = oracle_lib.OracleCrowd(osys, R)
    e_or, _ = orc.sweep(2)
    d = np.abs(gpu.qmc_get_positions() - orc.positions())
    same = np.all(np.minimum(d, wl.L - d) < 1e-9, axis=(1, 2))
    assert same.sum() >= wl.n_walkers - 1
    assert np.allclose(e2[:, same], e_or[:, same], rtol=1e-9, atol=1e-10)
    # taking the term out restores the plain local energy
    gpu.qmc_load_nlpp([], [], 0.0)
    e3 = np.zeros(wl.n_walkers)
    gpu.qmc_local_energy_batch(e3)
    plain = oracle_lib.OracleSystem(wl)
    Rg = gpu.qmc_get_positions()
    ref3 = np.array([plain.local_energy(Rg[w])[0] for w in range(wl.n_walkers)])
    assert np.allclose(e3, ref3, rtol=1e-10, atol=1e-10)


def test_nlpp_mixed_bench_geometry(Q, oracle_lib):
    """pw128 (32 ions) with the term on, 16 walkers after two mixed generations: E_L within
    the mixed path's 1e-3 of the oracle's FP64 recompute at the GPU's positions, with the
    nonlocal part well above that tolerance."""
    wl = wl_mod.pw128()
    W, rc = 16, 1.5
    gpu = Q.Crowd.from_workload(wl, precision="mixed", n_walkers=W)
    gpu.qmc_load_nlpp(AMPS, WIDTHS, rc)
    gpu.qmc_load_positions(np.ascontiguousarray(wl.positions(n_walkers=W)))
    gpu.qmc_recompute()
    e = np.zeros((2, W))
    gpu.qmc_sweep(2, e)
    Rg = gpu.qmc_get_positions()
    osys = oracle_lib.OracleSystem(wl, nlpp=(AMPS, WIDTHS, rc))
    big = 0
    for w in [0, 5, 11, 15]:
        ref = osys.local_energy(Rg[w])[0]
        tol = 1e-3 * max(1.0, abs(ref))
        assert abs(e[-1, w] - ref) < tol, (w, e[-1, w], ref)
        big += abs(osys.nlpp(Rg[w])) > 100 * tol
    assert big >= 2


def test_nlpp_arguments_and_batches(Q):
    wl = _ions26()
    c = Q.Crowd.from_workload(wl, precision="mixed")
    for amps, widths, rc in [((1.0,), (0.0,), 1.0), ((1.0,), (1.0,), 0.6 * wl.L),
                             ((1.0,) * 4, (1.0,) * 4, 1.0), ((1.0,), (1.0,), 0.0)]:
        with pytest.raises(Q.QmcError):
            c.qmc_load_nlpp(amps, widths, rc)
    c.qmc_load_nlpp((1.0,), (1.0,), 1.0)
    c2 = Q.Crowd.from_workload(wl, precision="mixed")
    with pytest.raises(Q.QmcError):
        Q.Batch([c, c2])


def test_nlpp_pair_list_overflow_matches_oracle(Q, oracle_lib):
    """A warp lists at most 64 (electron, ion) pairs within the cutoff for the CTA and
    evaluates the rest itself: 96 electrons (three per warp of the walker's 32), 64 ions and
    a cutoff of 0.45 L give some warps more than 64 pairs; E_L still equals the oracle's to
    1e-10 in FP64."""
    wl = wl_mod.make_workload("nl96", n_el=96, n_orb=48, grid=20, n_walkers=4, n_gen=1,
                              n_ions=64, tau=0.3, j1_knots=6, j2_knots=8)
    rc = 0.45 * wl.L
    R = np.ascontiguousarray(wl.positions())
    # pairs per warp (warp g takes electrons g, g + 32, g + 64), counted on the host
    d = R[:, :, None, :] - wl.ions[None, None, :, :]
    d -= wl.L * np.round(d / wl.L)
    within = (np.sqrt((d * d).sum(-1)) < rc).sum(-1)          # [W][N]
    per_warp = np.stack([within[:, g::32].sum(-1) for g in range(32)], axis=1)
    assert per_warp.max() > 64, per_warp.max()
    gpu = Q.Crowd.from_workload(wl, precision="fp64")
    gpu.qmc_load_nlpp(AMPS, WIDTHS, rc)
    gpu.qmc_load_positions(R)
    gpu.qmc_recompute()
    e = np.zeros(wl.n_walkers)
    gpu.qmc_local_energy_batch(e)
    osys = oracle_lib.OracleSystem(wl, nlpp=(AMPS, WIDTHS, rc))
    ref = np.array([osys.local_energy(R[w])[0] for w in range(wl.n_walkers)])
    assert np.allclose(e, ref, rtol=1e-10, atol=1e-10), np.abs(e - ref).max()
