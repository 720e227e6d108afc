"""Pins of the FP64 CPU oracle to facts outside itself (closed forms, exact reproduction,
brute force, finite differences, published known answers).  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2209_14487_gb300 import workloads as wl_mod

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- RNG
def test_philox_known_answers(oracle_lib):
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert list(oracle_lib.philox(w[:4], w[4:6])) == w[6:]
        n += 1
    assert n == 3


def test_move_draw_moments(oracle_lib):
    chis, us = [], []
    for w in range(4):
        for g in range(50):
            for i in range(100):
                chi, u = oracle_lib.move_draws(14487, w, g, i)
                chis.append(chi)
                us.append(u)
    chis = np.array(chis).ravel()
    us = np.array(us)
    n = chis.size
    assert abs(chis.mean()) < 4.0 / math.sqrt(n)
    assert abs(chis.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs((chis ** 4).mean() - 3.0) < 0.15
    assert us.min() > 0.0 and us.max() <= 1.0
    assert abs(us.mean() - 0.5) < 4.0 * math.sqrt(1.0 / 12.0 / us.size)
    # distinct walkers / generations / electrons give distinct streams
    a = oracle_lib.move_draws(1, 0, 0, 0)[0]
    for args in [(1, 1, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1), (2, 0, 0, 0)]:
        assert not np.allclose(a, oracle_lib.move_draws(*args)[0])


# ----------------------------------------------------------------------------- radial functor
def test_radial_partition_of_unity_and_linear_reproduction(oracle_lib):
    K, rc = 12, 3.0
    h = rc / K
    ones = np.ones(K)
    lin = np.arange(K, dtype=np.float64)
    for r in np.linspace(0.0, (K - 4) * h, 37):  # stencil i..i+3 inside the free coefficients
        u = oracle_lib.radial(ones, rc, r)
        assert abs(u[0] - 1.0) < 1e-14 and abs(u[1]) < 1e-12 and abs(u[2]) < 1e-10
        u = oracle_lib.radial(lin, rc, r)
        # sum_m (i+m) b_m(t) = i + t + 1 = r/h + 1
        assert abs(u[0] - (r / h + 1.0)) < 1e-12
        assert abs(u[1] - 1.0 / h) < 1e-11
        assert abs(u[2]) < 1e-9


def test_radial_cutoff_continuity_cusp(oracle_lib):
    wl = wl_mod.pw128()
    for jas, cusp in [(wl.j2_ud, -0.5), (wl.j2_uu, -0.25), (wl.j1, None)]:
        c, rc, K = jas.coefs, jas.rc, jas.K
        h = rc / K
        for r in [rc, rc + 1e-12, rc * 1.5]:
            assert np.all(oracle_lib.radial(c, rc, r) == 0.0)
        near = oracle_lib.radial(c, rc, rc * (1 - 1e-9))
        assert np.all(np.abs(near) < 1e-7)
        # C2 continuity across interior knots
        for i in range(1, K):
            lo = oracle_lib.radial(c, rc, i * h - 1e-10)
            hi = oracle_lib.radial(c, rc, i * h + 1e-10)
            assert np.allclose(lo, hi, atol=1e-7)
        if cusp is not None:
            assert abs(oracle_lib.radial(c, rc, 0.0)[1] - cusp) < 1e-13
        # derivatives against central differences
        for r in np.linspace(0.05, rc - 0.05, 23):
            e = 1e-5
            up, um, u0 = (oracle_lib.radial(c, rc, r + e), oracle_lib.radial(c, rc, r - e),
                          oracle_lib.radial(c, rc, r))
            assert abs((up[0] - um[0]) / (2 * e) - u0[1]) < 1e-7
            assert abs((up[1] - um[1]) / (2 * e) - u0[2]) < 1e-6


# ----------------------------------------------------------------------------- tricubic spline
def _poly_table(G, L, coef):
    """Coefficients c = prod_d (1 - h^2/6 d_d^2) p of a per-variable cubic
    p(x,y,z) = sum coef[a,b,c] x^a y^b z^c on the nodes; the spline of c equals p."""
    h = L / G
    x = np.arange(G) * h

    def pw(a, xs):
        return xs ** a

    def d2(a, xs):
        return a * (a - 1) * xs ** (a - 2) if a >= 2 else np.zeros_like(xs)

    T = np.zeros((G, G, G))
    for (a, b, c), v in np.ndenumerate(coef):
        fx = pw(a, x) - h * h / 6 * d2(a, x)
        fy = pw(b, x) - h * h / 6 * d2(b, x)
        fz = pw(c, x) - h * h / 6 * d2(c, x)
        T += v * fx[:, None, None] * fy[None, :, None] * fz[None, None, :]
    return T


def _poly_eval(coef, r):
    v = 0.0
    g = np.zeros(3)
    lap = 0.0
    x, y, z = r
    for (a, b, c), cf in np.ndenumerate(coef):
        px, py, pz = x ** a, y ** b, z ** c
        dx = a * x ** (a - 1) if a >= 1 else 0.0
        dy = b * y ** (b - 1) if b >= 1 else 0.0
        dz = c * z ** (c - 1) if c >= 1 else 0.0
        ddx = a * (a - 1) * x ** (a - 2) if a >= 2 else 0.0
        ddy = b * (b - 1) * y ** (b - 2) if b >= 2 else 0.0
        ddz = c * (c - 1) * z ** (c - 2) if c >= 2 else 0.0
        v += cf * px * py * pz
        g += cf * np.array([dx * py * pz, px * dy * pz, px * py * dz])
        lap += cf * (ddx * py * pz + px * ddy * pz + px * py * ddz)
    return v, g, lap


def test_spline_reproduces_cubic_polynomials(oracle_lib):
    G, L, n = 10, 3.0, 2
    rng = np.random.default_rng(7)
    coefs = [rng.standard_normal((4, 4, 4)) for _ in range(n)]
    table = np.stack([_poly_table(G, L, c) for c in coefs], axis=-1)
    osys = oracle_lib.OracleSystem(None, n_up=1, n_dn=1, n_orb=n, grid=G, L=L, table=table)
    h = L / G
    for _ in range(40):
        # cells 1..G-3 keep the 4-point stencil inside the nodes (no periodic wrap)
        r = rng.uniform(1.0 * h, (G - 2) * h - 1e-9, size=3)
        v, g, l = osys.spo_vgl(r, n)
        for j in range(n):
            pv, pg, pl = _poly_eval(coefs[j], r)
            scale = 1.0 + abs(pv)
            assert abs(v[j] - pv) < 1e-11 * scale * 50
            assert np.allclose(g[j], pg, rtol=1e-10, atol=1e-9)
            assert abs(l[j] - pl) < 1e-8 * (1 + abs(pl))


def test_spline_planewave_node_closed_forms(oracle_lib):
    wl = wl_mod.tiny(n_el=12, n_orb=6, grid=10, L=3.7)
    osys = oracle_lib.OracleSystem(wl)
    G, L = wl.grid, wl.L
    h = L / G
    rng = np.random.default_rng(3)
    for _ in range(12):
        gi = rng.integers(0, G, size=3)
        r = gi * h
        v, g, l = osys.spo_vgl(r)
        for j, terms in enumerate(wl.orbital_terms):
            ev = 0.0
            eg = np.zeros(3)
            el = 0.0
            for q, amp in terms:
                m, kind = wl.waves[q]
                k = 2 * np.pi * np.array(m) / L
                ph = float(k @ r)
                if kind == "1":
                    ev += amp
                    continue
                w, dw = (math.cos(ph), -math.sin(ph)) if kind == "c" else (math.sin(ph), math.cos(ph))
                fd = np.array([3 * math.sin(kd * h) / (h * (2 + math.cos(kd * h))) for kd in k])
                sd = np.array([3 * (2 * math.cos(kd * h) - 2) / (h * h * (2 + math.cos(kd * h)))
                               for kd in k])
                ev += amp * w
                eg += amp * fd * dw
                el += amp * sd.sum() * w
            assert abs(v[j] - ev) < 1e-12
            assert np.allclose(g[j], eg, atol=1e-11)
            assert abs(l[j] - el) < 1e-9


def test_spline_derivatives_match_central_differences(oracle_lib):
    wl = wl_mod.tiny(n_el=12, n_orb=6, grid=10, L=3.7)
    osys = oracle_lib.OracleSystem(wl)
    h = wl.L / wl.grid
    rng = np.random.default_rng(11)
    e = 1e-3 * h
    for _ in range(10):
        cell = rng.integers(0, wl.grid, size=3)
        r = (cell + rng.uniform(0.1, 0.9, size=3)) * h
        v0, g0, l0 = osys.spo_vgl(r)
        lap_fd = np.zeros_like(v0)
        for d in range(3):
            dr = np.zeros(3)
            dr[d] = e
            vp = osys.spo_vgl(r + dr)[0]
            vm = osys.spo_vgl(r - dr)[0]
            assert np.allclose((vp - vm) / (2 * e), g0[:, d], atol=1e-6)
            lap_fd += (vp - 2 * v0 + vm) / (e * e)
        assert np.allclose(lap_fd, l0, atol=2e-3)


# ----------------------------------------------------------------------------- determinants
def _leibniz(a):
    n = a.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        p = 1.0
        for i in range(n):
            p *= a[i, perm[i]]
        tot += (-1) ** inv * p
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_det_matches_leibniz(oracle_lib, n):
    rng = np.random.default_rng(n)
    for _ in range(3):
        a = rng.standard_normal((n, n))
        st, la, sg = oracle_lib.det(a)
        ref = _leibniz(a)
        assert st == 0
        assert sg == (1 if ref > 0 else -1)
        assert abs(la - math.log(abs(ref))) < 1e-12 * max(1.0, abs(la)) + 1e-13


def test_det_singular_and_inverse_identity(oracle_lib):
    a = np.ones((4, 4))
    assert oracle_lib.det(a)[0] == 1
    rng = np.random.default_rng(5)
    for n in [8, 64]:
        a = rng.standard_normal((n, n))
        st, inv, la, sg = oracle_lib.inverse(a)
        assert st == 0
        assert np.abs(inv @ a - np.eye(n)).max() < 1e-11
        assert np.abs(a @ inv - np.eye(n)).max() < 1e-11


# ----------------------------------------------------------------------------- wavefunction
def _tiny_crowd(oracle_lib, update=0, k=1, **kw):
    wl = wl_mod.tiny(**kw)
    osys = oracle_lib.OracleSystem(wl, update=update, delay_rank=k)
    R = wl.positions(n_walkers=wl.n_walkers)
    return wl, osys, R


def test_ratio_and_gradients_match_full_recompute(oracle_lib):
    wl, osys, R = _tiny_crowd(oracle_lib)
    crowd = oracle_lib.OracleCrowd(osys, R)
    rng = np.random.default_rng(21)
    for iel in [0, 3, 4, wl.n_el - 1]:
        rnew = np.mod(R[:, iel, :] + rng.normal(0, 0.4, size=(wl.n_walkers, 3)), wl.L)
        ratio, grad, lr, _ = crowd.propose(iel, rnew)
        for w in range(wl.n_walkers):
            la0, s0 = osys.logpsi(R[w])
            R1 = R[w].copy()
            R1[iel] = rnew[w]
            la1, s1 = osys.logpsi(R1)
            ref = s0 * s1 * math.exp(la1 - la0)
            assert abs(ratio[w] - ref) <= 1e-10 * abs(ref)
            assert abs(lr[w] - (la1 - la0)) < 1e-10 * max(1, abs(la1 - la0))
            # grad_i log|Psi| at R' by central differences of full recomputes
            e = 1e-5
            fd = np.zeros(3)
            for d in range(3):
                Rp = R1.copy(); Rp[iel, d] += e
                Rm = R1.copy(); Rm[iel, d] -= e
                fd[d] = (osys.logpsi(Rp)[0] - osys.logpsi(Rm)[0]) / (2 * e)
            assert np.allclose(grad[w], fd, rtol=1e-6, atol=1e-6)
        crowd.accept(iel, np.zeros(wl.n_walkers, dtype=np.uint8))
    g = crowd.eval_grad(2)
    for w in range(wl.n_walkers):
        e = 1e-5
        for d in range(3):
            Rp = R[w].copy(); Rp[2, d] += e
            Rm = R[w].copy(); Rm[2, d] -= e
            fd = (osys.logpsi(Rp)[0] - osys.logpsi(Rm)[0]) / (2 * e)
            assert abs(g[w, d] - fd) < 1e-6 * (1 + abs(fd))


def test_local_energy_matches_finite_differences(oracle_lib):
    wl, osys, R = _tiny_crowd(oracle_lib)
    h = 1e-4
    for w in range(2):
        e_l, grad, lap = osys.local_energy(R[w])
        la0, _ = osys.logpsi(R[w])
        kin = 0.0
        for i in range(wl.n_el):
            for d in range(3):
                Rp = R[w].copy(); Rp[i, d] += h
                Rm = R[w].copy(); Rm[i, d] -= h
                lp, sp = osys.logpsi(Rp)
                lm, sm = osys.logpsi(Rm)
                # Psi(R +- h)/Psi(R); signs do not change for a small step
                kin += (math.exp(lp - la0) + math.exp(lm - la0) - 2.0) / (h * h)
        ref = -0.5 * kin + osys.potential(R[w])
        assert abs(e_l - ref) < 2e-5 * max(1.0, abs(ref))


def test_delayed_update_equals_sherman_morrison(oracle_lib):
    res = {}
    for update, k in [(0, 1), (1, 3), (1, 4)]:
        wl, osys, R = _tiny_crowd(oracle_lib, update=update, k=k)
        crowd = oracle_lib.OracleCrowd(osys, R)
        rng = np.random.default_rng(99)
        seq = []
        # repeated rows inside one window: electron 1 moved three times, 2 twice
        for iel in [1, 2, 1, 0, 5, 1, 2, 6, 7, 3, 4, 0]:
            rnew = np.mod(R[:, iel, :] + rng.normal(0, 0.5, size=(wl.n_walkers, 3)), wl.L)
            ratio, grad, lr, _ = crowd.propose(iel, rnew)
            acc = (rng.uniform(size=wl.n_walkers) < 0.7).astype(np.uint8)
            crowd.accept(iel, acc)
            seq.append((ratio, grad))
        inv = [crowd.inverse(w, s) for w in range(wl.n_walkers) for s in range(2)]
        res[(update, k)] = (seq, inv, crowd.logpsi())
    base = res[(0, 1)]
    for key in [(1, 3), (1, 4)]:
        seq, inv, lp = res[key]
        for (r0, g0), (r1, g1) in zip(base[0], seq):
            assert np.allclose(r0, r1, rtol=1e-10, atol=0)
            assert np.allclose(g0, g1, rtol=1e-9, atol=1e-10)
        for a, b in zip(base[1], inv):
            assert np.allclose(a, b, rtol=1e-9, atol=1e-11)
        assert np.allclose(base[2][0], lp[0], rtol=1e-12)


def test_sweep_state_consistent_with_full_recompute(oracle_lib):
    wl, osys, R = _tiny_crowd(oracle_lib, n_walkers=3)
    crowd = oracle_lib.OracleCrowd(osys, R)
    e, na = crowd.sweep(3)
    assert na.sum() > 0
    Rn = crowd.positions()
    la, sg = crowd.logpsi()
    for w in range(3):
        ref, rs = osys.logpsi(Rn[w])
        assert abs(la[w] - ref) < 1e-10 * max(1, abs(ref))
        assert sg[w] == rs
        e_ref = osys.local_energy(Rn[w])[0]
        assert abs(e[-1, w] - e_ref) < 1e-9 * max(1, abs(e_ref))
        for s in range(2):
            A = crowd.A(w, s)
            B = crowd.inverse(w, s)
            assert np.abs(B @ A - np.eye(A.shape[0])).max() < 1e-10


def test_sweep_is_deterministic_and_counter_based(oracle_lib):
    wl, osys, R = _tiny_crowd(oracle_lib, n_walkers=3)
    c1 = oracle_lib.OracleCrowd(osys, R)
    c1.sweep(2)
    c2 = oracle_lib.OracleCrowd(osys, R)
    c2.sweep(1)
    c2.sweep(1)
    assert np.array_equal(c1.positions(), c2.positions())
    # a walker's trajectory does not depend on the other walkers of the crowd
    c3 = oracle_lib.OracleCrowd(osys, R[:2])
    c3.sweep(2)
    assert np.array_equal(c1.positions()[:2], c3.positions())


# ----------------------------------------------------------------------------- closed forms
def _free_electron(oracle_lib, n, L, W=5, analytic=True, G=16):
    waves = wl_mod.real_plane_waves(n)
    m = np.array([w[0] for w in waves], dtype=np.int32)
    kind = np.array([{"1": 0, "c": 1, "s": 2}[w[1]] for w in waves], dtype=np.int32)
    wl = wl_mod.make_workload("fe", n_el=2 * n, n_orb=n, grid=G, n_walkers=W, n_gen=1, L=L,
                              j2_knots=0, admix=0.0, potential=False)
    kw = {"analytic_waves": (m, kind)} if analytic else {}
    osys = oracle_lib.OracleSystem(wl, **kw)
    k2 = ((2 * np.pi / L) ** 2) * (m.astype(np.float64) ** 2).sum(axis=1)
    exact = 2 * 0.5 * k2.sum()   # both spins fill the same n waves
    return wl, osys, exact


def test_zero_variance_free_electrons(oracle_lib):
    wl, osys, exact = _free_electron(oracle_lib, n=7, L=4.3)
    R = wl.positions()
    es = [osys.local_energy(R[w])[0] for w in range(R.shape[0])]
    assert np.allclose(es, exact, rtol=1e-11, atol=1e-11)
    # through the crowd after moves: still the same constant
    crowd = oracle_lib.OracleCrowd(osys, R)
    e, na = crowd.sweep(2)
    assert np.allclose(e, exact, rtol=1e-10)


def test_spline_free_electron_energy_converges_second_order(oracle_lib):
    """Spline plane waves: lap phi + |k|^2 phi -> 0 as O(h^2) (cubic-spline second
    derivatives), and the free-electron E_L approaches sum |k|^2 / 2."""
    errs, emed = [], []
    waves = wl_mod.real_plane_waves(7)
    m = np.array([w[0] for w in waves], dtype=np.float64)
    for G in [12, 24, 48]:
        wl, osys, exact = _free_electron(oracle_lib, n=7, L=4.3, analytic=False, G=G)
        k2 = ((2 * np.pi / wl.L) ** 2) * (m ** 2).sum(axis=1)
        rng = np.random.default_rng(0)
        err = 0.0
        for _ in range(100):
            v, g, l = osys.spo_vgl(rng.uniform(0, wl.L, 3))
            err = max(err, np.abs(l + k2 * v).max())
        errs.append(err)
        R = wl.positions(n_walkers=24)
        e = np.array([osys.local_energy(R[w])[0] for w in range(R.shape[0])])
        emed.append(np.median(np.abs(e - exact)))
    for a, b in zip(errs, errs[1:]):
        assert 0.2 < b / a < 0.3
    assert emed[2] < emed[1] < emed[0]
    assert emed[2] < 1e-3 * exact


@pytest.mark.parametrize("drift,wave", [(0, 1), (1, 0), (2, 0), (1, 1)])
def test_metropolis_samples_psi_squared(oracle_lib, drift, wave):
    """One electron, Psi = w(x) exp(-u1) with w = cos(2 pi x / L) (with nodes) or w = 1
    (nodeless), moved by plain Metropolis (drift 0) or drift-diffusion Metropolis-Hastings
    with the limited drift (1) or the plain drift F (2): the walk's histogram on 4^3 bins
    against |Psi|^2 integrated on a fine grid (chi^2, p > 0.001).  A proposal density that
    the acceptance ratio does not match exactly (a wrong drift in either Green's function)
    biases the histogram."""
    from scipy import stats
    L = 3.0
    ions = np.array([[0.7, 1.1, 2.0], [2.2, 2.3, 0.6]])
    j1 = wl_mod.jastrow_coefs(6, -0.6, 1.4, cusp=None)
    m = np.array([[1, 0, 0] if wave else [0, 0, 0]], dtype=np.int32)
    kind = np.array([wave], dtype=np.int32)
    osys = oracle_lib.OracleSystem(None, analytic_waves=(m, kind), n_up=1, n_dn=0, n_orb=1,
                                   n_ions=2, ions=ions, j1_K=6, j1_rc=1.4, j1=j1.coefs, L=L,
                                   tau=0.4, drift=drift, seed=777)
    W, nb = 512, 4
    R = np.random.default_rng(1).uniform(0, L, size=(W, 1, 3))
    crowd = oracle_lib.OracleCrowd(osys, R)
    crowd.sweep(30)
    counts = np.zeros((nb, nb, nb))
    for _ in range(40):
        crowd.sweep(4)
        idx = np.minimum((crowd.positions()[:, 0, :] / L * nb).astype(int), nb - 1)
        np.add.at(counts, (idx[:, 0], idx[:, 1], idx[:, 2]), 1)
    f = 12
    xs = (np.arange(nb * f) + 0.5) * L / (nb * f)
    dens = np.zeros((nb * f,) * 3)
    for a, x in enumerate(xs):
        for b, y in enumerate(xs):
            for c, z in enumerate(xs):
                la, _ = osys.logpsi(np.array([[x, y, z]]))
                dens[a, b, c] = math.exp(2 * la)
    p = dens.reshape(nb, f, nb, f, nb, f).sum(axis=(1, 3, 5))
    p /= p.sum()
    exp_counts = p * counts.sum()
    chi2 = ((counts - exp_counts) ** 2 / exp_counts).sum()
    pval = stats.chi2.sf(chi2, nb ** 3 - 1)
    assert pval > 1e-3, (chi2, pval)


@pytest.mark.parametrize("drift,mx", [(1, 3), (2, 0), (0, 3)])
def test_drift_diffusion_samples_psi_squared_near_nodes(oracle_lib, drift, mx):
    """Sharper than the 4^3 histogram above: one electron in a 6 bohr cell with
    Psi = cos(2 pi mx x / L) exp(-u1) (mx = 3: six nodal planes; mx = 0: nodeless), moved
    with the limited drift (1), the plain drift F (2, nodeless only: near a node tau F
    outgrows the cell and the single-image Green's function no longer holds) or none
    (0); tau = 0.3.  The walk's 16-bin marginal in x against |Psi|^2 integrated over y and
    z (chi^2 with 15 degrees of freedom, p > 0.001; the RNG is counter-based, so the test
    is deterministic).  Near the nodes the limited and plain drifts differ most: an oracle
    whose reverse Green's function used F(r') instead of D(F(r')) gave chi^2 = 2049 here
    (p ~ 0), against 18.4 for the correct one."""
    from scipy import stats
    L, tau, nb = 6.0, 0.3, 16
    ions = np.array([[1.4, 2.2, 4.0], [4.4, 4.6, 1.2]])
    j1 = wl_mod.jastrow_coefs(6, -0.6, 1.4, cusp=None)
    m = np.array([[mx, 0, 0]], dtype=np.int32)
    kind = np.array([1], dtype=np.int32)
    osys = oracle_lib.OracleSystem(None, analytic_waves=(m, kind), n_up=1, n_dn=0, n_orb=1,
                                   n_ions=2, ions=ions, j1_K=6, j1_rc=1.4, j1=j1.coefs, L=L,
                                   tau=tau, drift=drift, seed=777)
    W = 1024
    R = np.random.default_rng(1).uniform(0, L, size=(W, 1, 3))
    crowd = oracle_lib.OracleCrowd(osys, R)
    crowd.sweep(30)
    counts = np.zeros(nb)
    for _ in range(40):
        crowd.sweep(8)
        idx = np.minimum((crowd.positions()[:, 0, 0] / L * nb).astype(int), nb - 1)
        np.add.at(counts, idx, 1)
    f, g = 8, 24
    xs = (np.arange(nb * f) + 0.5) * L / (nb * f)
    ys = (np.arange(g) + 0.5) * L / g
    dens = np.zeros(nb * f)
    for a, x in enumerate(xs):
        for y in ys:
            for z in ys:
                la, _ = osys.logpsi(np.array([[x, y, z]]))
                dens[a] += math.exp(2 * la)
    p = dens.reshape(nb, f).sum(axis=1)
    p /= p.sum()
    exp_counts = p * counts.sum()
    chi2 = ((counts - exp_counts) ** 2 / exp_counts).sum()
    pval = stats.chi2.sf(chi2, nb - 1)
    assert pval > 1e-3, (chi2, pval)


def test_potential_and_jastrow_pair_structure_closed_forms(oracle_lib):
    """Two electrons (opposite spins) and one ion in a large cell: V and U by hand."""
    L = 20.0
    j2 = wl_mod.jastrow_coefs(8, 0.5, 3.0, cusp=-0.5)
    j2l = wl_mod.jastrow_coefs(8, 0.5, 3.0, cusp=-0.25)
    j1 = wl_mod.jastrow_coefs(6, -0.3, 3.0, cusp=None)
    ions = np.array([[10.0, 10.0, 10.0]])
    osys = oracle_lib.OracleSystem(None, n_up=1, n_dn=1, n_orb=1, n_ions=1, ions=ions, L=L,
                                   potential=1, j2_K=8, j2_rc=3.0, j2_uu=j2l.coefs,
                                   j2_ud=j2.coefs, j1_K=6, j1_rc=3.0, j1=j1.coefs, grid=4,
                                   table=np.zeros((4, 4, 4, 1)))
    R = np.array([[10.0, 10.0, 11.2], [10.0, 9.3, 10.0]])
    r12 = math.sqrt(0.7 ** 2 + 1.2 ** 2)
    V = math.exp(-r12 ** 2) - 2 * math.exp(-0.5 * 1.2 ** 2) - 2 * math.exp(-0.5 * 0.7 ** 2)
    assert abs(osys.potential(R) - V) < 1e-14
    U = (oracle_lib.radial(j2.coefs, 3.0, r12)[0] + oracle_lib.radial(j1.coefs, 3.0, 1.2)[0]
         + oracle_lib.radial(j1.coefs, 3.0, 0.7)[0])
    assert abs(osys.jastrow_U(R) - U) < 1e-14
    # minimum image across the boundary and the L/2 truncation of V
    R2 = np.array([[0.2, 10.0, 10.0], [19.9, 10.0, 10.0]])
    ions2 = np.array([[0.0, 0.0, 0.0]])
    osys2 = oracle_lib.OracleSystem(None, n_up=1, n_dn=1, n_orb=1, n_ions=1, ions=ions2, L=L,
                                    potential=1, grid=4, table=np.zeros((4, 4, 4, 1)),
                                    j2_K=8, j2_rc=3.0, j2_uu=j2l.coefs, j2_ud=j2.coefs)
    assert abs(osys2.potential(R2) - math.exp(-0.3 ** 2)) < 1e-14  # ion beyond L/2 of both
    assert abs(osys2.jastrow_U(R2) - oracle_lib.radial(j2.coefs, 3.0, 0.3)[0]) < 1e-14


# ---- DMC reweighting and branching (Alg. 1 lines 13-14, readings of the scope table) ----

def test_dmc_branch_static_population_at_trial_energy(oracle_lib):
    """E_prev = E_new = E_T: every weight is 1 and floor(1 + u) = 1 for u in (0, 1), so the
    population is unchanged and in order."""
    e = np.full(37, -3.25)
    src, w = oracle_lib.dmc_branch(e, e, 16, 0.01, -3.25, 99, 4, 100)
    assert np.array_equal(src, np.arange(37))
    assert np.allclose(w, 1.0)


def test_dmc_branch_multiplicity_is_unbiased_and_ordered(oracle_lib):
    """floor(w + u) with u uniform has mean w: at weight 1.37 each walker leaves one or two
    copies, two with probability 0.37; copies of a walker are adjacent, walkers in order."""
    W, tau, et = 40000, 0.01, 0.0
    target = 1.37
    e = np.full(W, et - np.log(target) / tau)
    src, w = oracle_lib.dmc_branch(e, e, 32, tau, et, 2209, 7, 10 * W)
    assert np.allclose(w, target, rtol=1e-12)
    counts = np.bincount(src, minlength=W)
    assert set(np.unique(counts)) <= {1, 2}
    assert np.all(np.diff(src) >= 0)
    sigma = np.sqrt(0.37 * 0.63 / W)
    assert abs(len(src) / W - target) < 4 * sigma


def test_dmc_branch_weight_closed_form_and_cap(oracle_lib):
    rng = np.random.default_rng(4)
    ep, en = rng.normal(-2.0, 0.5, 10), rng.normal(-2.0, 0.5, 10)
    tau, et = 0.05, -1.7
    full, w = oracle_lib.dmc_branch(ep, en, 8, tau, et, 5, 2, 1000)
    assert np.allclose(w, np.exp(-tau * ((ep + en) / 2 - et)), rtol=1e-14)
    cut, _ = oracle_lib.dmc_branch(ep, en, 8, tau, et, 5, 2, 6)
    assert len(cut) == min(6, len(full))
    assert np.array_equal(cut, full[:len(cut)])


def test_dmc_zero_variance_population_is_static(oracle_lib):
    """Free electrons with analytic plane waves (no Jastrow, no potential): E_L is the
    constant sum |k|^2 / 2 at every fixed-node DMC step, so with E_T fed back from the
    weighted estimate every weight is 1 and the population stays the same walkers."""
    wl, _, exact = _free_electron(oracle_lib, n=7, L=4.3, W=12)
    waves = wl_mod.real_plane_waves(7)
    m = np.array([w[0] for w in waves], dtype=np.int32)
    kind = np.array([{"1": 0, "c": 1, "s": 2}[w[1]] for w in waves], dtype=np.int32)
    tau, W = 0.01, 12
    osys = oracle_lib.OracleSystem(wl, analytic_waves=(m, kind), dmc=1, tau=tau)
    crowd = oracle_lib.OracleCrowd(osys, wl.positions())
    e_prev = np.array(crowd.local_energy())
    e_trial = float(e_prev.mean())
    for g in range(6):
        e_new, na = crowd.sweep(1)
        assert na.sum() > 0
        assert np.allclose(e_new[0], exact, rtol=1e-10)
        src, w = oracle_lib.dmc_branch(e_prev, e_new[0], wl.n_el, tau, e_trial, wl.seed,
                                       crowd.generation - 1, 2 * W)
        assert np.array_equal(src, np.arange(W)), g
        assert np.allclose(w, 1.0, rtol=0, atol=1e-12)
        e_est = float((w * e_new[0]).sum() / w.sum())
        e_trial = e_est - 0.1 * np.log(len(src) / W) / tau
        e_prev = e_new[0][src]


def test_dmc_fixed_node_rejects_a_sign_change(oracle_lib):
    """A proposal whose determinant ratio is negative with rho^2 above the move's
    acceptance uniform u is accepted by plain Metropolis without drift (A = rho^2 > u) and
    rejected under the fixed-node rule."""
    wl = wl_mod.tiny(n_el=8, n_walkers=1, j1_knots=0, j2_knots=0)
    wl.drift = False
    R = wl.positions()
    plain = oracle_lib.OracleCrowd(oracle_lib.OracleSystem(wl), R)
    fixed = oracle_lib.OracleCrowd(oracle_lib.OracleSystem(wl, dmc=1), R)
    rng = np.random.default_rng(8)
    found = None
    for iel in range(wl.n_el):  # the electron with the smallest acceptance uniform first
        _, u = oracle_lib.move_draws(wl.seed, 0, plain.generation, iel)
        for _ in range(3000):
            rnew = rng.uniform(0.0, wl.L, size=(1, 3))
            ratio, _, _, _ = plain.propose(iel, rnew)
            plain.accept(iel, np.zeros(1, dtype=np.uint8))
            if ratio[0] < 0.0 and ratio[0] ** 2 > u:
                found = (iel, rnew)
                break
        if found:
            break
    assert found is not None
    iel, rnew = found
    plain.propose(iel, rnew)
    assert plain.accept(iel)[0] == 1
    fixed.propose(iel, rnew)
    assert fixed.accept(iel)[0] == 0


# ------------------------------------------------------------------ nonlocal pseudopotential
def test_nlpp_column_ratios_equal_full_recomputes(oracle_lib):
    """The nonlocal term from the inverse's columns (the fast form both the crowd and the
    CUDA path use) equals the one whose every ratio comes from two full recomputes of
    log|Psi| (Jastrow J1 + J2, both spins, three channels)."""
    wl = wl_mod.tiny(n_el=8, n_walkers=2, n_ions=3, L=4.0)
    osys = oracle_lib.OracleSystem(wl, nlpp=((0.8, -0.5, 0.3), (0.9, 1.1, 0.7), 1.6))
    R = wl.positions()
    n_pairs = 0
    for w in range(R.shape[0]):
        fast, slow = osys.nlpp(R[w]), osys.nlpp(R[w], direct=True)
        assert fast != 0.0
        assert abs(fast - slow) < 1e-10 * max(1.0, abs(slow))
        for i in range(wl.n_el):
            d = R[w, i] - wl.ions
            d -= wl.L * np.round(d / wl.L)
            n_pairs += int((np.linalg.norm(d, axis=1) < 1.6).sum())
    assert n_pairs >= 4
    # and the local energy carries it
    e_with = osys.local_energy(R[0])[0]
    e_without = oracle_lib.OracleSystem(wl).local_energy(R[0])[0]
    assert abs((e_with - e_without) - osys.nlpp(R[0])) < 1e-10 * max(1.0, abs(e_with))


def _one_wave_nlpp(oracle_lib, l, r):
    """One electron in a single real plane wave cos(k.x), one ion at distance r: the
    channel-l term against the exact sphere average (2l+1) Re(i^l e^{ik.c}) j_l(kr)
    P_l(d.k / (r k)) / cos(k.r_e), c the ion."""
    from scipy.special import eval_legendre, spherical_jn
    L = 6.0
    m = np.array([[1, 1, 0]], dtype=np.int32)
    kind = np.array([1], dtype=np.int32)
    k = 2 * np.pi / L * m[0].astype(float)
    wl = wl_mod.make_workload("one", n_el=2, n_orb=1, grid=8, n_walkers=1, n_gen=1, L=L,
                              j2_knots=0, admix=0.0, potential=False)
    ion = np.array([[2.1, 2.7, 3.0]])
    wl.ions = ion
    dirn = np.array([0.48, -0.6, 0.64])
    dirn /= np.linalg.norm(dirn)
    amps = [0.0, 0.0, 0.0]
    amps[l] = 1.0
    osys = oracle_lib.OracleSystem(wl, analytic_waves=(m, kind), n_up=1, n_dn=0, n_orb=1,
                                   nlpp=(amps[:l + 1], (1e6,) * (l + 1), 2.0))
    re = ion[0] + r * dirn
    got = osys.nlpp(re[None, :])
    kr = np.linalg.norm(k) * r
    phase = np.exp(1j * (k @ ion[0])) * (1j ** l)
    exact = ((2 * l + 1) * phase.real * spherical_jn(l, kr)
             * eval_legendre(l, dirn @ k / np.linalg.norm(k)) / np.cos(k @ re))
    return got, exact


@pytest.mark.parametrize("l,order", [(0, 6), (1, 5), (2, 4)])
def test_nlpp_channels_against_the_sphere_average(oracle_lib, l, order):
    """The 12-point rule is exact to degree 5: channel l misses the exact average by
    O((kr)^(6-l)), so halving r shrinks the error by about 2^(6-l); a wrong point set,
    weight, (2l+1), Legendre polynomial or sign of d would leave an O(1) error."""
    g1, x1 = _one_wave_nlpp(oracle_lib, l, 0.6)
    g2, x2 = _one_wave_nlpp(oracle_lib, l, 0.3)
    e1, e2 = abs(g1 - x1), abs(g2 - x2)
    assert abs(x1) > 1e-2 and abs(x2) > 1e-3
    assert e1 < 1e-2 * abs(x1)
    assert 0.5 * 2 ** order < e1 / e2 < 2.0 * 2 ** order, (e1, e2)


# ------------------------------------------------------------------ Ewald Coulomb energy
MADELUNG_NACL = 1.747564594633182  # rock salt, per ion pair in units of 1/d (d: nearest)


def _rock_salt(oracle_lib, L, alpha, mmax, shift=(0.0, 0.0, 0.0)):
    """The conventional rock-salt cell: 4 cations (+1, as ions) and 4 anions (-1, as
    electrons) at nearest-neighbour distance L/2."""
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    cat = np.mod((fcc + np.array(shift)) * L, L)
    an = np.mod((fcc + 0.5 + np.array(shift)) * L, L)
    osys = oracle_lib.OracleSystem(None, n_up=2, n_dn=2, n_orb=2, n_ions=4, L=L,
                                   ions=np.ascontiguousarray(cat), coul=1, coul_Z=1.0,
                                   coul_alpha=alpha, coul_mmax=mmax)
    return osys, np.ascontiguousarray(an)


def test_ewald_reproduces_the_rock_salt_madelung_constant(oracle_lib):
    L = 5.2
    for alpha, mmax in ((5.0 / L, 12), (7.0 / L, 16)):
        osys, R = _rock_salt(oracle_lib, L, alpha, mmax, shift=(0.13, 0.02, 0.31))
        E = osys.coulomb(R, images=True)
        assert abs(E - (-8.0 * MADELUNG_NACL / L)) < 1e-9, (alpha, E)


def test_ewald_is_independent_of_alpha_and_min_image_converges(oracle_lib):
    """The total does not depend on the splitting; with a large alpha the minimum-image
    real-space sum equals the 27-cell one."""
    rng = np.random.default_rng(3)
    L = 4.7
    osys, _ = _rock_salt(oracle_lib, L, 5.0 / L, 12)
    R = np.ascontiguousarray(rng.uniform(0, L, size=(4, 3)))
    ions = np.ascontiguousarray(rng.uniform(0, L, size=(4, 3)))
    ref = None
    for alpha, mmax in ((5.0 / L, 12), (6.5 / L, 15), (9.0 / L, 22)):
        o = oracle_lib.OracleSystem(None, n_up=2, n_dn=2, n_orb=2, n_ions=4, L=L, ions=ions,
                                    coul=1, coul_Z=1.0, coul_alpha=alpha, coul_mmax=mmax)
        e = o.coulomb(R, images=True)
        ref = e if ref is None else ref
        assert abs(e - ref) < 1e-9
    o = oracle_lib.OracleSystem(None, n_up=2, n_dn=2, n_orb=2, n_ions=4, L=L, ions=ions,
                                coul=1, coul_Z=1.0, coul_alpha=10.0 / L, coul_mmax=24)
    assert abs(o.coulomb(R, images=False) - ref) < 1e-8
    # a charged system: the background term keeps the total independent of alpha too
    e1 = oracle_lib.OracleSystem(None, n_up=2, n_dn=2, n_orb=2, n_ions=4, L=L, ions=ions,
                                 coul=1, coul_Z=2.0, coul_alpha=5.0 / L,
                                 coul_mmax=12).coulomb(R, images=True)
    e2 = oracle_lib.OracleSystem(None, n_up=2, n_dn=2, n_orb=2, n_ions=4, L=L, ions=ions,
                                 coul=1, coul_Z=2.0, coul_alpha=8.0 / L,
                                 coul_mmax=20).coulomb(R, images=True)
    assert abs(e1 - e2) < 1e-9
