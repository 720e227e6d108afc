"""The Ewald Coulomb term of E_L on the GPU (a kernel of its own after every E_L launch)
against the FP64 oracle (whose Ewald sum reproduces the rock-salt Madelung constant):
FP64 to 1e-10 for a charged and a neutral cell and through sweeps; mixed at the bench
geometry to 1e-4 of E_L; argument checks and the batch refusal."""
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


def _ions26():
    return wl_mod.make_workload("c26", n_el=26, n_orb=15, grid=14, n_walkers=7, n_gen=3,
                                n_ions=5, L=5.3, tau=0.4, j1_knots=7, j2_knots=9)


@pytest.mark.parametrize("Z", [26.0 / 5.0, 1.0])
def test_coulomb_fp64_matches_oracle(Q, oracle_lib, Z):
    wl = _ions26()
    alpha, mmax = 10.0 / wl.L, 12
    R = np.ascontiguousarray(wl.positions())
    gpu = Q.Crowd.from_workload(wl, precision="fp64")
    gpu.qmc_load_coulomb(Z, alpha, mmax)
    gpu.qmc_load_positions(R)
    gpu.qmc_recompute()
    e = np.zeros(wl.n_walkers)
    gpu.qmc_local_energy_batch(e)
    kw = dict(coul=1, coul_Z=Z, coul_alpha=alpha, coul_mmax=mmax)
    osys = oracle_lib.OracleSystem(wl, **kw)
    ref = np.array([osys.local_energy(R[w])[0] for w in range(wl.n_walkers)])
    vc = np.array([osys.coulomb(R[w]) for w in range(wl.n_walkers)])
    assert np.all(np.abs(vc) > 1.0)
    assert np.allclose(e, ref, rtol=1e-10, atol=1e-9)
    e2 = np.zeros((2, wl.n_walkers))
    gpu.qmc_sweep(2, e2)
    orc = oracle_lib.OracleCrowd(osys, R)
    e_or, _ = orc.sweep(2)
    d = np.abs(gpu.qmc_get_positions() - orc.positions())
    same = np.all(np.minimum(d, wl.L - d) < 1e-9, axis=(1, 2))
    assert same.sum() >= wl.n_walkers - 1
    assert np.allclose(e2[:, same], e_or[:, same], rtol=1e-9, atol=1e-9)
    gpu.qmc_load_coulomb(0.0, 1.0, 1, on=False)
    e3 = np.zeros(wl.n_walkers)
    gpu.qmc_local_energy_batch(e3)
    plain = oracle_lib.OracleSystem(wl)
    Rg = gpu.qmc_get_positions()
    assert np.allclose(e3, [plain.local_energy(Rg[w])[0] for w in range(wl.n_walkers)],
                       rtol=1e-10, atol=1e-10)


def test_coulomb_mixed_bench_geometry(Q, oracle_lib):
    """pw128 with Z = 4 on its 32 ions (a neutral cell), 16 walkers after two mixed
    generations."""
    wl = wl_mod.pw128()
    W, Z, alpha, mmax = 16, 4.0, 8.0 / wl.L, 10
    gpu = Q.Crowd.from_workload(wl, precision="mixed", n_walkers=W)
    gpu.qmc_load_coulomb(Z, alpha, mmax)
    gpu.qmc_load_positions(np.ascontiguousarray(wl.positions(n_walkers=W)))
    gpu.qmc_recompute()
    e = np.zeros((2, W))
    gpu.qmc_sweep(2, e)
    Rg = gpu.qmc_get_positions()
    osys = oracle_lib.OracleSystem(wl, coul=1, coul_Z=Z, coul_alpha=alpha, coul_mmax=mmax)
    for w in [0, 5, 11, 15]:
        ref = osys.local_energy(Rg[w])[0]
        assert abs(e[-1, w] - ref) < 1e-4 * abs(ref), (w, e[-1, w], ref)


def test_coulomb_arguments_and_batches(Q):
    wl = _ions26()
    c = Q.Crowd.from_workload(wl, precision="mixed")
    for Z, alpha, mmax in [(-1.0, 1.0, 4), (1.0, 0.0, 4), (1.0, 1.0, 0)]:
        with pytest.raises(Q.QmcError):
            c.qmc_load_coulomb(Z, alpha, mmax)
    with pytest.raises(Q.QmcError) as ei:
        c.qmc_load_coulomb(1.0, 1.0, 20)  # too many reciprocal vectors
    assert ei.value.status == Q.QMC_ERR_UNSUPPORTED
    c.qmc_load_coulomb(1.0, 2.0, 6)
    c2 = Q.Crowd.from_workload(wl, precision="mixed")
    with pytest.raises(Q.QmcError):
        Q.Batch([c, c2])
