"""DMC on the GPU (fixed-node moves, reweighting, branching with the walkers' full state
copied on the device) against the FP64 oracle: identical populations, positions and
local energies generation by generation."""
import numpy as np
import pytest

from paper_2209_14487_gb300 import workloads as wl_mod

pytestmark = pytest.mark.gpu

TAU = 0.01


@pytest.fixture(scope="module")
def Q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14487_gb300 import qmcgb
    return qmcgb


def _system():
    # 16 electrons, 4 ions, J1 + J2, the DMC time step
    return wl_mod.make_workload("dmc16", n_el=16, n_orb=8, grid=20, n_walkers=24, n_gen=4,
                                n_ions=4, L=5.0, tau=TAU, j1_knots=6, j2_knots=8)


@pytest.mark.parametrize("update,k", [("sm", 1), ("delayed", 3)])
def test_dmc_fp64_generations_match_oracle(Q, oracle_lib, update, k):
    wl = _system()
    W = wl.n_walkers
    R = np.ascontiguousarray(wl.positions())
    gpu = Q.Crowd.from_workload(wl, precision="fp64", update=update, delay_rank=k, dmc=True)
    gpu.qmc_load_positions(R)
    gpu.qmc_recompute()
    osys = oracle_lib.OracleSystem(wl, dmc=1, update=1 if update == "delayed" else 0,
                                   delay_rank=k)
    orc = oracle_lib.OracleCrowd(osys, R)
    e_prev = np.zeros(W)
    gpu.qmc_local_energy_batch(e_prev)
    assert np.allclose(e_prev, orc.local_energy(), rtol=1e-10)
    e_trial = float(e_prev.mean())
    for g in range(4):
        Wg = gpu.W
        e_new = np.zeros((1, Wg))
        gpu.qmc_sweep(1, e_new)
        e_or, _ = orc.sweep(1)
        assert np.allclose(e_new[0], e_or[0], rtol=1e-9, atol=1e-12), g
        st, e_next = gpu.qmc_dmc_branch(e_prev, e_new[0], e_trial)
        src, wts = oracle_lib.dmc_branch(e_prev, e_or[0], wl.n_el, TAU, e_trial, wl.seed,
                                         orc.generation - 1, W)
        assert st.n_before == Wg and st.n_after == len(src), (g, st.n_after, len(src))
        assert np.isclose(st.w_sum, wts.sum(), rtol=1e-12)
        assert np.isclose(st.we_sum, (wts * e_or[0]).sum(), rtol=1e-9)
        R_or = orc.positions()[src]
        assert np.allclose(gpu.qmc_get_positions(), R_or, atol=1e-12, rtol=0), g
        assert np.allclose(e_next, e_or[0][src], rtol=1e-9)
        la, sg = gpu.qmc_get_logpsi()
        gen = orc.generation
        orc = oracle_lib.OracleCrowd(osys, np.ascontiguousarray(R_or))
        orc.generation = gen
        ola, osg = orc.logpsi()
        assert np.allclose(la, ola, rtol=1e-9) and np.array_equal(sg, osg)
        e_prev = e_next
        e_trial = float(st.we_sum / st.w_sum)


def test_dmc_fixed_node_on_the_gpu(Q, oracle_lib):
    """The fine-grained accept with the internal Metropolis test: a proposal with a
    negative determinant ratio and rho^2 above u is accepted by a plain crowd and rejected
    by a DMC crowd."""
    wl = wl_mod.tiny(n_el=8, n_walkers=1, j1_knots=0, j2_knots=0)
    wl.drift = False
    R = np.ascontiguousarray(wl.positions())
    probe = oracle_lib.OracleCrowd(oracle_lib.OracleSystem(wl), R)
    rng = np.random.default_rng(8)
    found = None
    for iel in range(wl.n_el):
        _, u = oracle_lib.move_draws(wl.seed, 0, 0, iel)
        for _ in range(3000):
            rnew = rng.uniform(0.0, wl.L, size=(1, 3))
            ratio, _, _, _ = probe.propose(iel, rnew)
            probe.accept(iel, np.zeros(1, dtype=np.uint8))
            if ratio[0] < 0.0 and ratio[0] ** 2 > u:
                found = (iel, rnew)
                break
        if found:
            break
    assert found is not None
    iel, rnew = found
    for dmc, expect in ((False, 1), (True, 0)):
        c = Q.Crowd.from_workload(wl, precision="fp64", dmc=dmc)
        c.qmc_load_positions(R)
        c.qmc_recompute()
        c.qmc_propose_move_batch(iel, np.ascontiguousarray(rnew))
        out = np.zeros(1, dtype=np.uint8)
        c.qmc_accept_reject_batch(iel, None, out)
        assert out[0] == expect, dmc


def test_dmc_mixed_population_control(Q):
    """Mixed precision, 40 generations with the trial-energy feedback of the readings:
    the population stays near its target inside the capacity and energies stay finite."""
    wl = wl_mod.pw128()
    cap, target = 96, 64
    c = Q.Crowd.from_workload(wl, precision="mixed", n_walkers=cap, dmc=True, tau=TAU)
    c.qmc_load_positions(np.ascontiguousarray(wl.positions(n_walkers=cap)))
    c.qmc_recompute()
    e_prev = np.zeros(cap)
    c.qmc_local_energy_batch(e_prev)
    e_trial = float(e_prev.mean())
    sizes = []
    for g in range(40):
        e_new = np.zeros((1, c.W))
        c.qmc_sweep(1, e_new)
        assert np.all(np.isfinite(e_new))
        st, e_prev = c.qmc_dmc_branch(e_prev, e_new[0], e_trial)
        sizes.append(st.n_after)
        e_est = st.we_sum / st.w_sum
        e_trial = e_est - np.log(st.n_after / target) / TAU * 0.1
    assert c.walker_count == sizes[-1] == c.W
    assert 0.5 * target <= np.mean(sizes[-10:]) <= cap, sizes


@pytest.mark.parametrize("precision,update,k", [("fp64", "sm", 1), ("mixed", "delayed", 8)])
def test_select_and_append_walkers(Q, oracle_lib, precision, update, k):
    """qmc_dmc_select keeps walkers src in order with their whole state; qmc_dmc_append adds
    walkers whose rows and inverses are built on arrival, leaving the others untouched.
    The FP64 crowd then sweeps exactly as an oracle crowd started from its positions."""
    wl = _system()
    gpu = Q.Crowd.from_workload(wl, precision=precision, update=update, delay_rank=k,
                                dmc=True)
    gpu.qmc_load_positions(np.ascontiguousarray(wl.positions()))
    gpu.qmc_recompute()
    gpu.qmc_sweep(1, np.zeros((1, gpu.W)))
    R1 = gpu.qmc_get_positions()
    la1, sg1 = gpu.qmc_get_logpsi()
    src = [5, 5, 0, 17, 3, 22, 9]
    gpu.qmc_dmc_select(src)
    assert gpu.W == gpu.walker_count == len(src)
    R2 = gpu.qmc_get_positions()
    la2, sg2 = gpu.qmc_get_logpsi()
    assert np.array_equal(R2, R1[src])
    assert np.array_equal(la2, la1[src]) and np.array_equal(sg2, sg1[src])
    # bad requests change nothing
    for bad in ([0, 7], [-1]):
        with pytest.raises(Q.QmcError):
            gpu.qmc_dmc_select(bad)
    with pytest.raises(Q.QmcError):
        gpu.qmc_dmc_append(np.zeros((wl.n_walkers, wl.n_el, 3)))
    assert gpu.walker_count == len(src)
    Rn = np.ascontiguousarray(wl.positions(crowd_id=3, n_walkers=5))
    gpu.qmc_dmc_append(Rn)
    assert gpu.W == gpu.walker_count == 12
    R3 = gpu.qmc_get_positions()
    la3, sg3 = gpu.qmc_get_logpsi()
    assert np.array_equal(R3[:7], R2) and np.array_equal(la3[:7], la2)
    assert np.allclose(R3[7:], np.mod(Rn, wl.L), rtol=0, atol=1e-12)
    osys = oracle_lib.OracleSystem(wl, dmc=1, update=1 if update == "delayed" else 0,
                                   delay_rank=k)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for w in range(7, 12):
        ref, rs = osys.logpsi(R3[w])
        assert abs(la3[w] - ref) <= tol * max(1.0, abs(ref)) and sg3[w] == rs
    if precision == "fp64":
        gen = gpu.generation
        e = np.zeros((1, 12))
        gpu.qmc_sweep(1, e)
        orc = oracle_lib.OracleCrowd(osys, np.ascontiguousarray(R3))
        orc.generation = gen
        e_or, _ = orc.sweep(1)
        assert np.allclose(e, e_or, rtol=1e-9)
        assert np.allclose(gpu.qmc_get_positions(), orc.positions(), rtol=0, atol=1e-12)
