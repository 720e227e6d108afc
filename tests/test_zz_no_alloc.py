"""The allocation-free inverse (qmc_inverse_noalloc) against the crowd's own FP64
recompute on the same Slater matrices, through the C ABI, on two calls in a row.

It serves callers that must not allocate device memory when they need an inverse
(host callbacks, latency-critical loops, runtimes that own all device memory), so its
workspace is a static device array shared by every call.  This file is collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_inverse_noalloc_matches_crowd_recompute():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14487_gb300 import qmcgb, workloads
    # no Jastrow, no ions: log|Psi| = log|det A_up| + log|det A_dn|
    wl = workloads.make_workload("noalloc", n_el=128, n_orb=64, grid=48, n_walkers=96,
                                 n_gen=1, L=10.0, j2_knots=0)
    crowd = qmcgb.Crowd.from_workload(wl, precision="fp64")
    crowd.qmc_load_positions(np.ascontiguousarray(wl.positions()))
    crowd.qmc_recompute()
    logpsi, sgn = crowd.qmc_get_logpsi()
    W, n = wl.n_walkers, wl.n_up
    ld_sum = np.zeros(W)
    sg_prod = np.ones(W, dtype=np.int64)
    for spin in (0, 1):   # two calls in a row on the shared static workspace
        A = crowd.qmc_get_slater_matrix(spin)
        ref = crowd.qmc_get_inverse(spin)
        a = torch.from_numpy(A).cuda()
        inv = torch.empty_like(a)
        ld = torch.empty(W, dtype=torch.float64, device="cuda")
        sg = torch.empty(W, dtype=torch.int32, device="cuda")
        qmcgb.qmc_inverse_noalloc(a, inv, ld, sg)
        torch.cuda.synchronize()
        got = inv.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
        eye = np.einsum("wij,wjk->wik", got, A)
        assert np.abs(eye - np.eye(n)).max() < 1e-9
        ld_sum += ld.cpu().numpy()
        sg_prod *= sg.cpu().numpy()
    assert np.allclose(ld_sum, logpsi, rtol=1e-12, atol=1e-10)
    assert np.array_equal(sg_prod, sgn)


def test_inverse_noalloc_limits_and_singular():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14487_gb300 import qmcgb
    a = torch.zeros((2, 3, 3), dtype=torch.float64, device="cuda")
    a[0] = torch.eye(3, dtype=torch.float64) * 2.0
    inv = torch.empty_like(a)
    ld = torch.empty(2, dtype=torch.float64, device="cuda")
    sg = torch.empty(2, dtype=torch.int32, device="cuda")
    qmcgb.qmc_inverse_noalloc(a, inv, ld, sg)
    torch.cuda.synchronize()
    assert np.allclose(inv[0].cpu().numpy(), np.eye(3) * 0.5)
    assert abs(ld[0].item() - 3 * np.log(2.0)) < 1e-14 and sg[0].item() == 1
    assert sg[1].item() == 0 and ld[1].item() == -np.inf
    big = torch.zeros((1, 1025, 1025), dtype=torch.float64, device="cuda")
    with pytest.raises(qmcgb.QmcError) as ei:
        qmcgb.qmc_inverse_noalloc(big, torch.empty_like(big), ld[:1], sg[:1])
    assert ei.value.status == 8


def test_inverse_noalloc_several_launches():
    """A batch larger than the static workspace holds (2^21 doubles: 8 matrices of 512 x 512)
    runs as several launches in stream order on the reused workspace: 9 matrices, two
    launches, each inverse, log|det| and sign against numpy."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14487_gb300 import qmcgb
    n, batch = 512, 9
    rng = np.random.default_rng(7)
    A = rng.normal(size=(batch, n, n)) + 4.0 * np.sqrt(n) * np.eye(n) * rng.choice([-1.0, 1.0],
                                                                               size=(batch, 1, 1))
    a = torch.from_numpy(A).cuda()
    inv = torch.empty_like(a)
    ld = torch.empty(batch, dtype=torch.float64, device="cuda")
    sg = torch.empty(batch, dtype=torch.int32, device="cuda")
    for _ in range(2):   # two calls in a row on the shared workspace
        qmcgb.qmc_inverse_noalloc(a, inv, ld, sg)
        torch.cuda.synchronize()
        got = inv.cpu().numpy()
        ref = np.linalg.inv(A)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
        s_ref, l_ref = np.linalg.slogdet(A)
        assert np.allclose(ld.cpu().numpy(), l_ref, rtol=1e-12, atol=1e-9)
        assert np.array_equal(sg.cpu().numpy(), s_ref.astype(np.int32))
