"""The move kernel's two shared-memory layouts through the C ABI.  Compact (the delayed
window's new orbital rows kept in global memory, each move's draws computed from the same
Philox words when needed) changes where operands live, not the arithmetic, so both layouts
give the same trajectories bit for bit on the same sweep path; compact also lets the FP64 path run the
1536-electron system, whose draw table does not fit in shared memory, checked here against
the oracle's trajectory."""
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


def _run(Q, wl, W, layout, n_gen, **kw):
    c = Q.Crowd.from_workload(wl, n_walkers=W, layout=layout, **kw)
    assert c.kernel_config["layout"] == layout, c.kernel_config
    c.qmc_load_positions(np.ascontiguousarray(wl.positions(n_walkers=W)))
    c.qmc_recompute()
    e = np.zeros((n_gen, W))
    st = c.qmc_sweep(n_gen, e)
    la, sg = c.qmc_get_logpsi()
    out = (c.qmc_get_positions(), e, la, sg, st.n_accept)
    c.close()
    return out


@pytest.mark.parametrize("make,kw", [
    (wl_mod.pw512, dict(precision="mixed", update="delayed", delay_rank=32, cta_threads=128)),
    (wl_mod.pw512, dict(precision="mixed", update="delayed", delay_rank=16, cta_threads=256)),
    # (the incremental Sherman-Morrison sweep of small systems pipelines its proposals and
    # needs the draw table, so a compact pw128 crowd takes the plain sweep: another path)
    (wl_mod.pw512, dict(precision="mixed", update="sm", cta_threads=256)),
    (wl_mod.pw128, dict(precision="fp64", update="delayed", delay_rank=4, cta_threads=128)),
])
def test_compact_layout_equals_shared(Q, make, kw):
    wl = make()
    a = _run(Q, wl, 16, "shared", 2, **kw)
    b = _run(Q, wl, 16, "compact", 2, **kw)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_dmc1536_layout_picks(Q):
    """The library's pick at n = 768: shared for the mixed delayed kernel (compact would
    fit two 128-thread CTAs on an SM, measured slower: the window's rows then come from
    L2 on every move); FP64 Sherman-Morrison fits only compact."""
    wl = wl_mod.dmc1536()
    m = Q.Crowd.from_workload(wl, precision="mixed", update="delayed", delay_rank=32,
                              cta_threads=128, n_walkers=2)
    assert m.kernel_config["layout"] == "shared", m.kernel_config
    mc = Q.Crowd.from_workload(wl, precision="mixed", update="delayed", delay_rank=32,
                               cta_threads=128, n_walkers=2, layout="compact")
    cfg = mc.kernel_config
    assert cfg["layout"] == "compact" and 2 * (cfg["smem_bytes"] + 1024) <= 228 * 1024, cfg
    d = Q.Crowd.from_workload(wl, precision="fp64", cta_threads=128, n_walkers=2)
    assert d.kernel_config["layout"] == "compact", d.kernel_config
    with pytest.raises(Q.QmcError) as ei:
        Q.Crowd.from_workload(wl, precision="fp64", cta_threads=128, n_walkers=2,
                              layout="shared")
    assert ei.value.status == Q.QMC_ERR_UNSUPPORTED


def test_fp64_dmc1536_follows_oracle(Q, oracle_lib):
    """FP64 Sherman-Morrison on the 1536-electron system (compact layout): one generation
    of two walkers on the internal RNG follows the oracle's trajectory (every decision the
    same; positions to 1e-8 bohr in a 22.9 bohr cell, the rounding of 1536 FP64 moves
    whose drifts the GPU sums in another order) and E_L to 1e-9."""
    wl = wl_mod.dmc1536()
    W = 2
    R = np.ascontiguousarray(wl.positions(n_walkers=W))
    gpu = Q.Crowd.from_workload(wl, precision="fp64", cta_threads=128, n_walkers=W,
                                n_recompute=0)
    gpu.qmc_load_positions(R)
    gpu.qmc_recompute()
    e = np.zeros((1, W))
    st = gpu.qmc_sweep(1, e)
    orc = oracle_lib.OracleCrowd(oracle_lib.OracleSystem(wl), R)
    e_or, na = orc.sweep(1)
    Rg, Ro = gpu.qmc_get_positions(), orc.positions()
    d = np.abs(Rg - Ro)
    d = np.minimum(d, wl.L - d)
    assert d.max() < 1e-8, d.max()
    assert st.n_accept == int(na.sum())
    assert np.allclose(e, e_or, rtol=1e-9, atol=1e-9), (e, e_or)
