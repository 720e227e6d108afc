"""The benchmark's own kernel path move by move against the oracle: the mixed
Sherman-Morrison sweep of the 128-electron system (incremental Jastrow, the pipelined next
electron's drift from three gathered sums, the FP64-exact Metropolis decision), and its
VMC energy against the FP64 path's after equilibration (Alg. 1 lines 5-11)."""
import math

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


def _move_bound(oracle_lib, seed, w, i, tau, fnorm):
    """Bound on |r'_GPU - r'_oracle| for one move from one configuration: the mixed path
    draws its Box-Muller radii sqrt(-2 ln u) from 24-bit uniforms of the same Philox words
    (|du| <= 2^-24, so |dr| <= 2^-24 / (u r)) and forms the drift in FP32 from the sweep's
    updated inverse and incremental Jastrow sums (|dF| <= 5e-5 (1 + |F|); a fresh FP32 drift
    is good to ~1e-6); the angles and the rest cost a few FP32 ulps."""
    key = [seed & 0xFFFFFFFF, (w ^ (seed >> 32)) & 0xFFFFFFFF]
    dchi = 0.0
    for slot in (0, 1):
        x = oracle_lib.philox([0, i, slot, 0], key)
        u = (((int(x[0]) >> 5) << 26) + (int(x[1]) >> 6) + 0.5) * 2.0 ** -53
        r = np.sqrt(-2.0 * np.log(u))
        dchi += 2.0 ** -24 / (u * r) + 1e-6 * r
    return np.sqrt(tau) * dchi + tau * 5e-5 * (1.0 + fnorm) + 1e-8


def test_mixed_sweep_follows_oracle_move_by_move(Q, oracle_lib):
    """One generation of 8 walkers on the internal counter-based RNG, checked move by move:
    before its move i a walker's configuration is known exactly (electrons j < i where the
    sweep left them, the others where they started), so the oracle takes move i from that
    same configuration (drift, proposal, ratio, Metropolis-Hastings test in FP64).  The
    GPU's decision (recorded per move) must equal the oracle's except where the FP32
    acceptance lies within rounding of the uniform (none expected in 1024 moves; at most 2
    allowed), and every accepted electron must sit at the oracle's proposal within one
    move's FP32 error (_move_bound).  E_L at the final positions equals the oracle's to
    1e-4."""
    wl = wl_mod.pw128()
    W, N = 8, wl.n_el
    R0 = np.ascontiguousarray(wl.positions(n_walkers=W))
    gpu = Q.Crowd.from_workload(wl, precision="mixed", update="sm", n_walkers=W,
                                n_recompute=0, cta_threads=128)
    gpu.qmc_load_positions(R0)
    gpu.qmc_recompute()
    gpu.qmc_trace_accepts(True)
    e = np.zeros((1, W))
    st = gpu.qmc_sweep(1, e)
    dec_gpu = gpu.qmc_get_accept_trace()
    Rg = gpu.qmc_get_positions()
    assert int(dec_gpu.sum()) == st.n_accept

    osys = oracle_lib.OracleSystem(wl)
    orc = oracle_lib.OracleCrowd(osys, R0)
    flips, worst = 0, 0.0
    for i in range(N):
        cfg = R0.copy()
        cfg[:, :i] = Rg[:, :i]
        orc.set_positions(cfg)
        assert orc.recompute() == 0
        orc.generation = 0
        F = orc.eval_grad(i)
        _, _, _, rnew = orc.propose(i)
        dec = orc.accept(i)
        flips += int(np.sum(dec != dec_gpu[:, i]))
        for w in np.nonzero((dec == 1) & (dec_gpu[:, i] == 1))[0]:
            d = np.abs(Rg[w, i] - rnew[w])
            d = float(np.minimum(d, wl.L - d).max())
            bound = _move_bound(oracle_lib, wl.seed, w, i, wl.tau, np.linalg.norm(F[w]))
            assert d <= bound, (w, i, d, bound)
            worst = max(worst, d / bound)
        # a rejected move leaves the electron where it was (to the 32-bit fixed point)
        rej = dec_gpu[:, i] == 0
        assert np.allclose(Rg[rej, i], R0[rej, i], rtol=0, atol=1e-8)
    e_or = np.array([osys.local_energy(Rg[w])[0] for w in range(W)])
    print(f"decisions that differ: {flips} of {W * N}; largest position difference of an "
          f"accepted move / its bound {worst:.2f}; acceptance {dec_gpu.mean():.3f}")
    assert flips <= 2
    assert np.all(np.abs(e[0] - e_or) < 1e-4 * np.maximum(1.0, np.abs(e_or))), (e[0], e_or)
    assert 0.5 < dec_gpu.mean() < 0.95


def _blocked_mean(e, n_block):
    m = e.mean(axis=1)                       # per-generation crowd average
    b = m[: len(m) // n_block * n_block].reshape(-1, n_block).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(len(b))


def test_mixed_vmc_energy_matches_fp64_at_pw128(Q):
    """VMC at the benchmark's configuration (256 walkers, 128 electrons): 60 generations of
    equilibration, then 120 generations in blocks of 10; the mixed path's energy lies
    within 2 sigma of the FP64 path's (sigma from the blocks of both runs)."""
    wl = wl_mod.pw128()
    burn, n_gen, blk = 60, 120, 10
    R0 = np.ascontiguousarray(wl.positions())
    res = {}
    for prec in ("fp64", "mixed"):
        c = Q.Crowd.from_workload(wl, precision=prec)
        c.qmc_load_positions(R0)
        c.qmc_recompute()
        c.qmc_sweep(burn)
        e = np.zeros((n_gen, wl.n_walkers))
        c.qmc_sweep(n_gen, e)
        res[prec] = _blocked_mean(e, blk)
        c.close()
    (m64, s64), (m32, s32) = res["fp64"], res["mixed"]
    print(f"E fp64 {m64:.4f} +- {s64:.4f}, mixed {m32:.4f} +- {s32:.4f}")
    assert abs(m64 - m32) < 2.0 * math.hypot(s64, s32), res
