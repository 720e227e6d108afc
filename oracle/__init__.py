"""ctypes wrapper of the plain FP64 CPU oracle (oracle/qmc_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg use it; the product path never imports it.  The C source shares nothing
with the CUDA path.  `build()` compiles it with gcc (-O3, OpenMP over walkers as in the
paper's Alg. 2); the library is rebuilt when the source is newer.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp,
                        _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class System(C.Structure):
    _fields_ = [
        ("n_up", C.c_int), ("n_dn", C.c_int), ("n_orb", C.c_int), ("n_ions", C.c_int),
        ("grid", C.c_int), ("drift", C.c_int), ("potential", C.c_int), ("update", C.c_int),
        ("delay_rank", C.c_int), ("n_recompute", C.c_int), ("j2_K", C.c_int),
        ("j1_K", C.c_int), ("analytic", C.c_int), ("dmc", C.c_int),
        ("L", C.c_double), ("tau", C.c_double), ("j2_rc", C.c_double), ("j1_rc", C.c_double),
        ("seed", C.c_uint64),
        ("table", C.c_void_p), ("ions", C.c_void_p), ("j2_uu", C.c_void_p),
        ("j2_ud", C.c_void_p), ("j1", C.c_void_p), ("pw_m", C.c_void_p),
        ("pw_kind", C.c_void_p),
        ("nl_n", C.c_int), ("nl_pad", C.c_int), ("nl_rc", C.c_double),
        ("nl_a", C.c_double * 3), ("nl_s", C.c_double * 3),
        ("coul", C.c_int), ("coul_mmax", C.c_int), ("coul_alpha", C.c_double),
        ("coul_Z", C.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        L.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_move_draws.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p,
                                    C.c_void_p]
        L.or_radial.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_void_p]
        L.or_spo_vgl.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]
        L.or_jastrow_U.argtypes = [C.c_void_p, C.c_void_p]
        L.or_jastrow_U.restype = C.c_double
        L.or_potential.argtypes = [C.c_void_p, C.c_void_p]
        L.or_potential.restype = C.c_double
        L.or_det.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.or_inverse.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_logpsi.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_local_energy.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]
        L.or_crowd_create.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.or_crowd_create.restype = C.c_void_p
        L.or_crowd_destroy.argtypes = [C.c_void_p]
        L.or_crowd_recompute.argtypes = [C.c_void_p]
        L.or_crowd_flush.argtypes = [C.c_void_p]
        L.or_crowd_eval_grad.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.or_crowd_propose.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
        L.or_crowd_accept.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.or_crowd_local_energy.argtypes = [C.c_void_p, C.c_void_p]
        L.or_crowd_sweep.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        L.or_crowd_get_positions.argtypes = [C.c_void_p, C.c_void_p]
        L.or_crowd_set_positions.argtypes = [C.c_void_p, C.c_void_p]
        L.or_crowd_get_logpsi.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_crowd_get_inverse.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.or_crowd_get_A.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
        L.or_crowd_get_generation.argtypes = [C.c_void_p]
        L.or_crowd_get_generation.restype = C.c_uint32
        L.or_crowd_set_generation.argtypes = [C.c_void_p, C.c_uint32]
        L.or_num_threads.restype = C.c_int
        L.or_coulomb.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
        L.or_coulomb.restype = C.c_double
        L.or_nlpp.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
        L.or_nlpp.restype = C.c_double
        L.or_set_num_threads.argtypes = [C.c_int]
        L.or_dmc_branch.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                    C.c_double, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p,
                                    C.c_void_p]
        L.or_dmc_branch.restype = C.c_int
        del dp
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class OracleSystem:
    """An or_system plus the numpy arrays it points into (kept alive here)."""

    def __init__(self, wl=None, *, update: int = 0, delay_rank: int = 1, analytic_waves=None,
                 n_recompute: int | None = None, seed: int | None = None, **override):
        s = System()
        self._keep = []
        if wl is not None:
            s.n_up, s.n_dn, s.n_orb = wl.n_up, wl.n_dn, wl.n_orb
            s.n_ions, s.grid = wl.n_ions, wl.grid
            s.drift, s.potential = int(wl.drift), int(wl.potential)
            s.L, s.tau = wl.L, wl.tau
            s.seed = wl.seed if seed is None else seed
            s.n_recompute = wl.n_recompute if n_recompute is None else n_recompute
            if analytic_waves is None:
                self.table = np.ascontiguousarray(wl.table(), dtype=np.float64)
                s.table = _p(self.table)
            self.ions = np.ascontiguousarray(wl.ions.reshape(-1, 3), dtype=np.float64)
            s.ions = _p(self.ions) if wl.n_ions else None
            if wl.j2_uu is not None:
                self.j2_uu = np.ascontiguousarray(wl.j2_uu.coefs)
                self.j2_ud = np.ascontiguousarray(wl.j2_ud.coefs)
                s.j2_K, s.j2_rc = wl.j2_uu.K, wl.j2_uu.rc
                s.j2_uu, s.j2_ud = _p(self.j2_uu), _p(self.j2_ud)
            if wl.j1 is not None:
                self.j1 = np.ascontiguousarray(wl.j1.coefs)
                s.j1_K, s.j1_rc = wl.j1.K, wl.j1.rc
                s.j1 = _p(self.j1)
        s.update, s.delay_rank = update, delay_rank
        if analytic_waves is not None:
            m, kind = analytic_waves
            self.pw_m = np.ascontiguousarray(m, dtype=np.int32)
            self.pw_kind = np.ascontiguousarray(kind, dtype=np.int32)
            s.analytic = 1
            s.pw_m, s.pw_kind = _p(self.pw_m), _p(self.pw_kind)
        nlpp = override.pop("nlpp", None)
        if nlpp is not None:  # (amplitudes a_l, widths s_l, cutoff): channels l = 0..
            amps, widths, rc = nlpp
            s.nl_n, s.nl_rc = len(amps), float(rc)
            s.nl_a = (C.c_double * 3)(*amps)
            s.nl_s = (C.c_double * 3)(*widths)
        for k, v in override.items():
            if isinstance(v, np.ndarray):
                self._keep.append(v)
                v = _p(v)
            setattr(s, k, v)
        self.s = s

    @property
    def ref(self):
        return C.byref(self.s)

    @property
    def n_el(self) -> int:
        return self.s.n_up + self.s.n_dn

    # ---- whole-configuration quantities ----
    def spo_vgl(self, r, n: int | None = None):
        n = self.s.n_orb if n is None else n
        r = np.ascontiguousarray(r, dtype=np.float64)
        v = np.zeros(n); g = np.zeros((n, 3)); l = np.zeros(n)
        lib().or_spo_vgl(self.ref, _p(r), n, _p(v), _p(g), _p(l))
        return v, g, l

    def logpsi(self, R):
        R = np.ascontiguousarray(R, dtype=np.float64)
        la = C.c_double(); sg = C.c_int()
        st = lib().or_logpsi(self.ref, _p(R), C.byref(la), C.byref(sg))
        if st:
            raise ZeroDivisionError("singular Slater matrix")
        return la.value, sg.value

    def jastrow_U(self, R):
        R = np.ascontiguousarray(R, dtype=np.float64)
        return lib().or_jastrow_U(self.ref, _p(R))

    def potential(self, R):
        R = np.ascontiguousarray(R, dtype=np.float64)
        return lib().or_potential(self.ref, _p(R))

    def coulomb(self, R, images: bool = False) -> float:
        """The Ewald Coulomb energy at R (minimum-image or 27-cell real-space sum)."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        return lib().or_coulomb(self.ref, _p(R), int(images))

    def nlpp(self, R, direct: bool = False) -> float:
        """The nonlocal term of E_L at R: ratios from full recomputes of log|Psi|
        (direct) or from the inverse's columns."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        return lib().or_nlpp(self.ref, _p(R), int(direct))

    def local_energy(self, R):
        """(E_L, grad log Psi [N][3], lap log Psi [N]) by full recompute."""
        R = np.ascontiguousarray(R, dtype=np.float64)
        N = self.n_el
        g = np.zeros((N, 3)); l = np.zeros(N); e = C.c_double()
        st = lib().or_local_energy(self.ref, _p(R), _p(g), _p(l), C.byref(e))
        if st:
            raise ZeroDivisionError("singular Slater matrix")
        return e.value, g, l


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def move_draws(seed: int, walker: int, gen: int, iel: int):
    chi = np.zeros(3); u = C.c_double()
    lib().or_move_draws(seed, walker, gen, iel, _p(chi), C.byref(u))
    return chi, u.value


def radial(coefs, rc: float, r: float):
    c = np.ascontiguousarray(coefs, dtype=np.float64)
    out = np.zeros(3)
    lib().or_radial(_p(c), c.shape[0], rc, r, _p(out))
    return out


def det(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    la = C.c_double(); sg = C.c_int()
    st = lib().or_det(_p(a), a.shape[0], C.byref(la), C.byref(sg))
    return st, la.value, sg.value


def inverse(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    inv = np.zeros_like(a)
    la = C.c_double(); sg = C.c_int()
    st = lib().or_inverse(_p(a), a.shape[0], _p(inv), C.byref(la), C.byref(sg))
    return st, inv, la.value, sg.value


class OracleCrowd:
    """W walkers of one system, driven through the same calls as the batched API."""

    def __init__(self, osys: OracleSystem, R):
        self.osys = osys
        R = np.ascontiguousarray(R, dtype=np.float64)
        self.W, self.N = R.shape[0], R.shape[1]
        self.h = lib().or_crowd_create(osys.ref, self.W, _p(R))
        st = lib().or_crowd_recompute(self.h)
        if st:
            raise ZeroDivisionError("singular Slater matrix at start")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_crowd_destroy(h)
            self.h = None

    def recompute(self):
        return lib().or_crowd_recompute(self.h)

    def flush(self):
        lib().or_crowd_flush(self.h)

    def eval_grad(self, iel):
        g = np.zeros((self.W, 3))
        lib().or_crowd_eval_grad(self.h, iel, _p(g))
        return g

    def propose(self, iel, rnew=None):
        ratio = np.zeros(self.W); grad = np.zeros((self.W, 3)); lr = np.zeros(self.W)
        rout = np.zeros((self.W, 3))
        rp = None
        if rnew is not None:
            rnew = np.ascontiguousarray(rnew, dtype=np.float64)
            rp = _p(rnew)
        lib().or_crowd_propose(self.h, iel, rp, _p(ratio), _p(grad), _p(lr), _p(rout))
        return ratio, grad, lr, rout

    def accept(self, iel, accept=None):
        out = np.zeros(self.W, dtype=np.uint8)
        ap = None
        if accept is not None:
            accept = np.ascontiguousarray(accept, dtype=np.uint8)
            ap = _p(accept)
        st = lib().or_crowd_accept(self.h, iel, ap, _p(out))
        if st:
            raise RuntimeError("accept without a pending proposal for this electron")
        return out

    def local_energy(self):
        e = np.zeros(self.W)
        lib().or_crowd_local_energy(self.h, _p(e))
        return e

    def sweep(self, n_gen):
        e = np.zeros((n_gen, self.W)); na = np.zeros(self.W, dtype=np.int64)
        st = lib().or_crowd_sweep(self.h, n_gen, _p(e), _p(na))
        if st:
            raise ZeroDivisionError("singular Slater matrix at a recompute")
        return e, na

    def positions(self):
        R = np.zeros((self.W, self.N, 3))
        lib().or_crowd_get_positions(self.h, _p(R))
        return R

    def set_positions(self, R):
        R = np.ascontiguousarray(R, dtype=np.float64)
        lib().or_crowd_set_positions(self.h, _p(R))

    def logpsi(self):
        la = np.zeros(self.W); sg = np.zeros(self.W, dtype=np.int32)
        lib().or_crowd_get_logpsi(self.h, _p(la), _p(sg))
        return la, sg

    def inverse(self, w, spin):
        ns = self.osys.s.n_up if spin == 0 else self.osys.s.n_dn
        out = np.zeros((ns, ns))
        lib().or_crowd_get_inverse(self.h, w, spin, _p(out))
        return out

    def A(self, w, spin):
        ns = self.osys.s.n_up if spin == 0 else self.osys.s.n_dn
        out = np.zeros((ns, ns))
        lib().or_crowd_get_A(self.h, w, spin, _p(out))
        return out

    @property
    def generation(self):
        return lib().or_crowd_get_generation(self.h)

    @generation.setter
    def generation(self, g):
        lib().or_crowd_set_generation(self.h, g)


def dmc_branch(e_prev, e_new, n_el: int, tau: float, e_trial: float, seed: int, gen: int,
               cap: int):
    """DMC reweighting and branching (or_dmc_branch): (src walker of every new slot,
    weights)."""
    e_prev = np.ascontiguousarray(e_prev, dtype=np.float64)
    e_new = np.ascontiguousarray(e_new, dtype=np.float64)
    W = e_prev.size
    src = np.zeros(max(cap, 1), dtype=np.int32)
    wt = np.zeros(W)
    n = lib().or_dmc_branch(_p(e_prev), _p(e_new), W, n_el, tau, e_trial, seed, gen, cap,
                            _p(src), _p(wt))
    return src[:n].copy(), wt


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops over walkers from now on."""
    lib().or_set_num_threads(int(n))
