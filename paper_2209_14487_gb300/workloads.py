"""Seeded synthetic workloads for the particle-by-particle move over a crowd of walkers.

This module only *makes inputs*: cells, ions, initial electron positions, the tricubic
B-spline coefficient table of synthetic plane-wave orbitals, and radial Jastrow
coefficients.  It evaluates no wavefunction, ratio, update or energy, so the CUDA path
and the CPU oracle can both be fed from it without sharing any of the method's
arithmetic.

The paper (Luo, Doak, Kent, arXiv:2209.14487) benchmarks NiO supercells (Sec. IV, Fig. 6)
whose orbitals and pseudopotentials are not available here.  The recipe below stands in
for them with tables of the same shapes and sizes:

* electrons: closed shell, N/2 up then N/2 down; one orbital set shared by both spins;
* cell: periodic cube of side L; where a workload gives no L, the density of the
  128-electron L=10 cell is kept, L = 5 (N/16)^(1/3);
* orbital j = w_j + sum_{m=1..3} a_jm w_{q_jm}: the j-th real plane wave plus three
  admixtures drawn uniformly from the first 2n real waves with a_jm ~ 0.3 N(0,1);
  real plane waves are 1, cos(k.r), sin(k.r), k in (2 pi / L) Z^3, ordered by |k|;
* the table holds, per wave, the periodic cubic B-spline interpolation coefficients of
  that wave on the G^3 grid (the wave at the node times prod_d 3/(2 + cos(k_d h))),
  summed over the orbital's terms; layout [G][G][G][n] (x slowest, orbital fastest);
* radial Jastrow: K coefficients c_m = a (1 - m/K)^2 (a = 0.5 for J2, -0.3 for J1) with
  the electron-electron cusp imposed on c_0 (u'(0) = -1/2 unlike, -1/4 like spins);
* ions and initial electrons are uniform in the cell.

Seeds: system 2209, walkers 14487 + crowd id.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SYSTEM_SEED = 2209
WALKER_SEED = 14487


@dataclass
class Jastrow:
    """Radial cubic B-spline functor input: K free coefficients and cutoff rc."""

    coefs: np.ndarray  # (K,) float64
    rc: float

    @property
    def K(self) -> int:
        return int(self.coefs.shape[0])


@dataclass
class Workload:
    name: str
    n_up: int
    n_dn: int
    n_orb: int
    grid: int
    L: float
    n_walkers: int
    n_gen: int
    tau: float
    n_recompute: int
    ions: np.ndarray                     # (NI, 3)
    j2_uu: Jastrow | None
    j2_ud: Jastrow | None
    j1: Jastrow | None
    waves: list = field(default_factory=list)      # [(m (3 ints), kind 'c'|'s'|'1')]
    orbital_terms: list = field(default_factory=list)  # per orbital [(wave index, amplitude)]
    drift: bool = True
    potential: bool = True
    seed: int = WALKER_SEED
    _table: np.ndarray | None = None

    @property
    def n_el(self) -> int:
        return self.n_up + self.n_dn

    @property
    def n_ions(self) -> int:
        return int(self.ions.shape[0])

    def table(self) -> np.ndarray:
        """Coefficient table [G][G][G][n_orb] float64 (built once, cached)."""
        if self._table is None:
            self._table = spline_table(self.grid, self.waves, self.orbital_terms)
        return self._table

    def positions(self, crowd_id: int = 0, n_walkers: int | None = None) -> np.ndarray:
        W = self.n_walkers if n_walkers is None else n_walkers
        rng = np.random.default_rng(WALKER_SEED + crowd_id)
        return rng.uniform(0.0, self.L, size=(W, self.n_el, 3))


def real_plane_waves(count: int) -> list:
    """The first `count` real plane waves on the integer lattice, ordered by |m|^2.

    Each entry is (m, kind) with kind '1' (constant), 'c' (cos) or 's' (sin); for each
    lattice vector m in the half space (first non-zero component positive) the cos
    wave precedes the sin wave.  Ties in |m|^2 are broken by the tuple m.
    """
    M = 1
    while True:
        rng_ = range(-M, M + 1)
        ms = []
        for a in rng_:
            for b in rng_:
                for c in rng_:
                    m = (a, b, c)
                    if m == (0, 0, 0):
                        continue
                    first = next(x for x in m if x != 0)
                    if first > 0:
                        ms.append(m)
        ms.sort(key=lambda m: (m[0] * m[0] + m[1] * m[1] + m[2] * m[2], m))
        waves = [((0, 0, 0), "1")]
        for m in ms:
            waves.append((m, "c"))
            waves.append((m, "s"))
        # the cube [-M, M]^3 holds every m with |m|^2 <= M^2; make sure the cut is inside it
        if len(waves) >= count:
            cut = waves[count - 1][0]
            if cut[0] ** 2 + cut[1] ** 2 + cut[2] ** 2 <= M * M:
                return waves[:count]
        M += 1


def orbital_terms(n: int, n_waves_pool: int, rng: np.random.Generator, admix: float = 0.3,
                  n_admix: int = 3) -> list:
    """Per orbital j: [(j, 1.0)] plus `n_admix` seeded admixtures from the first pool waves."""
    terms = []
    for j in range(n):
        t = [(j, 1.0)]
        qs = rng.integers(0, n_waves_pool, size=n_admix)
        amps = admix * rng.standard_normal(n_admix)
        for q, a in zip(qs, amps):
            if admix != 0.0:
                t.append((int(q), float(a)))
        terms.append(t)
    return terms


def spline_table(G: int, waves: list, terms: list) -> np.ndarray:
    """Periodic cubic B-spline coefficients of the orbitals on a G^3 grid.

    For a real plane wave with integer vector m the interpolating coefficients are the
    wave's node values times prod_d 3 / (2 + cos(2 pi m_d / G)); k_d h = 2 pi m_d / G does
    not depend on L.  Returns float64 [G][G][G][n].
    """
    n = len(terms)
    out = np.zeros((n, G, G, G), dtype=np.float64)  # orbital-major while accumulating
    th = 2.0 * np.pi * np.arange(G) / G
    for j, tlist in enumerate(terms):
        # sum over terms of separable products: cos(x+y+z) = c_xy cos z - s_xy sin z and
        # sin(x+y+z) = s_xy cos z + c_xy sin z, one (G^2 x 2T) (2T x G) product per orbital
        xy = np.zeros((G, G, 2 * len(tlist)))
        zz = np.zeros((2 * len(tlist), G))
        for t, (q, amp) in enumerate(tlist):
            m, kind = waves[q]
            if kind == "1":
                xy[:, :, 2 * t] = 1.0
                zz[2 * t] = amp
                continue
            fac = 1.0
            for d in range(3):
                fac *= 3.0 / (2.0 + math.cos(2.0 * math.pi * m[d] / G))
            a = m[0] * th[:, None] + m[1] * th[None, :]
            cxy, sxy = np.cos(a), np.sin(a)
            cz, sz = amp * fac * np.cos(m[2] * th), amp * fac * np.sin(m[2] * th)
            xy[:, :, 2 * t], xy[:, :, 2 * t + 1] = cxy, sxy
            if kind == "c":
                zz[2 * t], zz[2 * t + 1] = cz, -sz
            else:
                zz[2 * t], zz[2 * t + 1] = sz, cz
        out[j] = (xy.reshape(G * G, -1) @ zz).reshape(G, G, G)
    return np.ascontiguousarray(np.moveaxis(out, 0, -1))


def jastrow_coefs(K: int, a: float, rc: float, cusp: float | None) -> Jastrow:
    """c_m = a (1 - m/K)^2; with `cusp` set, c_0 = c_2 - 2 h cusp so u'(0) = cusp."""
    c = np.array([a * (1.0 - m / K) ** 2 for m in range(K)], dtype=np.float64)
    if cusp is not None:
        h = rc / K
        c[0] = c[2] - 2.0 * h * cusp
    return Jastrow(coefs=c, rc=float(rc))


def make_workload(name: str, n_el: int, n_orb: int, grid: int, n_walkers: int, n_gen: int,
                  n_ions: int = 0, L: float | None = None, tau: float = 0.5,
                  n_recompute: int = 0, j1_knots: int = 0, j2_knots: int = 10,
                  admix: float = 0.3, potential: bool = True, drift: bool = True,
                  crowd_seed_offset: int = 0) -> Workload:
    if L is None:
        L = 5.0 * (n_el / 16.0) ** (1.0 / 3.0)
    n_up = n_el // 2
    n_dn = n_el - n_up
    rng = np.random.default_rng(SYSTEM_SEED)
    waves = real_plane_waves(max(2 * n_orb, n_orb + 1))
    terms = orbital_terms(n_orb, 2 * n_orb, rng, admix=admix)
    ion_rng = np.random.default_rng(SYSTEM_SEED + 1)
    ions = ion_rng.uniform(0.0, L, size=(n_ions, 3)) if n_ions > 0 else np.zeros((0, 3))
    j2_uu = j2_ud = j1 = None
    if j2_knots > 0:
        rc2 = min(L / 2.0, 2.5)
        j2_uu = jastrow_coefs(j2_knots, 0.5, rc2, cusp=-0.25)
        j2_ud = jastrow_coefs(j2_knots, 0.5, rc2, cusp=-0.5)
    if j1_knots > 0 and n_ions > 0:
        rc1 = min(L / 2.0, 3.0)
        j1 = jastrow_coefs(j1_knots, -0.3, rc1, cusp=None)
    return Workload(name=name, n_up=n_up, n_dn=n_dn, n_orb=n_orb, grid=grid, L=float(L),
                    n_walkers=n_walkers, n_gen=n_gen, tau=tau, n_recompute=n_recompute,
                    ions=ions, j2_uu=j2_uu, j2_ud=j2_ud, j1=j1, waves=waves,
                    orbital_terms=terms, drift=drift, potential=potential,
                    seed=WALKER_SEED + crowd_seed_offset)


def pw16() -> Workload:
    """16 electrons (8/8), L = 5, 8 orbitals on 32^3, J2 10 knots rc = 2.5, 16 walkers,
    100 sweeps, tau = 0.5, Sherman-Morrison update, FP64."""
    return make_workload("pw16_fp64_sm", n_el=16, n_orb=8, grid=32, n_walkers=16, n_gen=100,
                         L=5.0, tau=0.5, n_recompute=0, j2_knots=10)


def pw128() -> Workload:
    """128 electrons (64/64), 64 orbitals on 48^3, 32 ions in L = 10 with J1 (8 knots) and
    J2 (10 knots), 256 walkers, 200 sweeps, FP64 recompute every 64 sweeps."""
    return make_workload("pw128_j1j2", n_el=128, n_orb=64, grid=48, n_walkers=256, n_gen=200,
                         n_ions=32, L=10.0, tau=0.5, n_recompute=64, j1_knots=8, j2_knots=10)


def pw512() -> Workload:
    """512 electrons (256/256), 256 orbitals on 64^3, no ions, J2, 1024 walkers."""
    return make_workload("pw512_j2", n_el=512, n_orb=256, grid=64, n_walkers=1024, n_gen=256,
                         tau=0.5, n_recompute=128, j2_knots=10)


def _mixed_size(n_el: int, n_orb: int, grid: int, n_walkers: int, offset: int) -> Workload:
    # the density of pw16/pw128 (L = 5 (N/16)^(1/3)), N/4 ions, J1 (8 knots) + J2 (10)
    return make_workload(f"mix{n_el}", n_el=n_el, n_orb=n_orb, grid=grid, n_walkers=n_walkers,
                         n_gen=200, n_ions=n_el // 4, tau=0.5, n_recompute=64, j1_knots=8,
                         j2_knots=10, crowd_seed_offset=offset)


def mix64() -> Workload:
    """64 electrons (32/32), 32 orbitals on 32^3, 16 ions, L = 7.94, 512 walkers."""
    return _mixed_size(64, 32, 32, 512, 0)


def mix192() -> Workload:
    """192 electrons (96/96), 96 orbitals on 48^3, 48 ions, L = 11.45, 256 walkers."""
    return _mixed_size(192, 96, 48, 256, 1)


def mix384() -> Workload:
    """384 electrons (192/192), 192 orbitals on 64^3, 96 ions, L = 14.42, 128 walkers."""
    return _mixed_size(384, 192, 64, 128, 2)


MIXED_BATCH = (mix64, mix192, mix384)


def dmc1536() -> Workload:
    """1536 electrons (768/768), 768 orbitals on 96^3, 64 ions, L = 22.9, J1 (8 knots) and
    J2 (10), 512 walkers, DMC time step 0.01, FP64 recompute every 128 generations."""
    return make_workload("dmc1536", n_el=1536, n_orb=768, grid=96, n_walkers=512, n_gen=100,
                         n_ions=64, tau=0.01, n_recompute=128, j1_knots=8, j2_knots=10)

WORKLOADS = {"pw16": pw16, "pw128": pw128, "pw512": pw512, "mix64": mix64, "mix192": mix192,
             "mix384": mix384, "dmc1536": dmc1536}


def tiny(n_el: int = 8, n_orb: int | None = None, grid: int = 12, n_walkers: int = 4,
         n_ions: int = 3, L: float = 4.0, j1_knots: int = 6, j2_knots: int = 8,
         admix: float = 0.3, potential: bool = True, drift: bool = True,
         tau: float = 0.3) -> Workload:
    """Small systems for oracle pins and quick parity cases."""
    if n_orb is None:
        n_orb = (n_el + 1) // 2
    return make_workload(f"tiny{n_el}", n_el=n_el, n_orb=n_orb, grid=grid, n_walkers=n_walkers,
                         n_gen=2, n_ions=n_ions, L=L, tau=tau, n_recompute=0,
                         j1_knots=j1_knots, j2_knots=j2_knots, admix=admix,
                         potential=potential, drift=drift)
