"""Python binding of libqmcgb (include/qmcgb.h): argument marshalling only.

Every computation runs in the CUDA library.  Host arrays (numpy, or CPU torch tensors) are
passed with QMC_MEM_HOST, CUDA torch tensors with QMC_MEM_DEVICE; one call's buffers must
all live on the same side.  There is no CPU fallback: without the compiled library,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# QMCGB_CHECK=1 in the environment selects the bounds-checked build of the same sources
CHECKED = os.environ.get("QMCGB_CHECK", "0") == "1"
LIB_PATH = os.path.join(HERE, "libqmcgb_check.so" if CHECKED else "libqmcgb.so")

QMC_OK = 0
QMC_ERR_UNSUPPORTED = 8
QMC_ERR_BOUNDS = 9
QMC_BUILD_CHECKED = 1
CHECK_SITES = {1: "walker", 2: "electron", 3: "spline cell", 4: "stencil item", 5: "window count",
               6: "shared-memory layout", 7: "stencil copy", 8: "pair-list ion",
               9: "DMC source walker"}
QMC_MEM_HOST, QMC_MEM_DEVICE = 0, 1
QMC_PREC_FP64, QMC_PREC_MIXED = 0, 1
QMC_UPDATE_SM, QMC_UPDATE_DELAYED = 0, 1
QMC_J1, QMC_J2_UU, QMC_J2_UD = 0, 1, 2
QMC_DTYPE_F64, QMC_DTYPE_F32 = 0, 1
QMC_STAGING_AUTO, QMC_STAGING_LDG = 0, 1
QMC_ENGINE_AUTO, QMC_ENGINE_SIMT = 0, 1
QMC_LAYOUT_AUTO, QMC_LAYOUT_SHARED, QMC_LAYOUT_COMPACT = 0, 1, 2
LAYOUTS = {"auto": QMC_LAYOUT_AUTO, "shared": QMC_LAYOUT_SHARED, "compact": QMC_LAYOUT_COMPACT}
GUARD_TOL_DEFAULT = 0.1  # the library's inverse-guard bound (run.guard_tol = 0)
STATUS_NAMES = {0: "QMC_OK", 1: "QMC_ERR_INVALID_ARG", 2: "QMC_ERR_OOM", 3: "QMC_ERR_CUDA",
                4: "QMC_ERR_SINGULAR", 5: "QMC_ERR_TIMEOUT", 6: "QMC_ERR_NAN",
                7: "QMC_ERR_STATE", 8: "QMC_ERR_UNSUPPORTED", 9: "QMC_ERR_BOUNDS"}

# every symbol include/qmcgb.h declares
EXPORTS = [
    "qmc_crowd_create", "qmc_crowd_destroy", "qmc_load_positions", "qmc_load_ions",
    "qmc_load_orbitals", "qmc_load_jastrow", "qmc_recompute", "qmc_eval_grad_batch",
    "qmc_propose_move_batch", "qmc_accept_reject_batch", "qmc_local_energy_batch", "qmc_sweep",
    "qmc_get_positions", "qmc_get_logpsi", "qmc_get_inverse", "qmc_get_slater_matrix",
    "qmc_get_generation", "qmc_set_generation", "qmc_get_launch_count", "qmc_crowd_save",
    "qmc_crowd_restore", "qmc_status_string", "qmc_inverse_noalloc", "qmc_get_kernel_config",
    "qmc_last_cuda_error", "qmc_batch_create", "qmc_batch_destroy", "qmc_batch_sweep",
    "qmc_batch_get_launch_count", "qmc_dmc_branch", "qmc_get_walker_count", "qmc_dmc_select",
    "qmc_dmc_append", "qmc_load_nlpp", "qmc_load_coulomb", "qmc_get_update", "qmc_get_guard",
    "qmc_trace_accepts", "qmc_get_accept_trace", "qmc_test_skip_stencil_copy",
    "qmc_build_flags", "qmc_check_report", "qmc_test_plant_bad_cell",
]


class qmc_system_desc(C.Structure):
    _fields_ = [("n_up", C.c_int), ("n_dn", C.c_int), ("n_orb", C.c_int), ("n_ions", C.c_int),
                ("grid", C.c_int), ("reserved", C.c_int), ("L", C.c_double)]


class qmc_run_desc(C.Structure):
    _fields_ = [("n_walkers", C.c_int), ("precision", C.c_int), ("update", C.c_int),
                ("delay_rank", C.c_int), ("n_recompute", C.c_int), ("drift", C.c_int),
                ("potential", C.c_int), ("staging", C.c_int), ("tau", C.c_double),
                ("seed", C.c_uint64), ("cta_threads", C.c_int), ("engine", C.c_int),
                ("dmc", C.c_int), ("layout", C.c_int), ("guard_tol", C.c_double)]


class qmc_dmc_stats(C.Structure):
    _fields_ = [("n_before", C.c_int), ("n_after", C.c_int), ("n_wanted", C.c_longlong),
                ("w_sum", C.c_double), ("we_sum", C.c_double)]


class qmc_stats(C.Structure):
    _fields_ = [("e_sum", C.c_double), ("e2_sum", C.c_double), ("n_samples", C.c_longlong),
                ("n_accept", C.c_longlong), ("n_moves", C.c_longlong),
                ("n_repair", C.c_longlong)]


class QmcError(RuntimeError):
    def __init__(self, fn: str, status: int, detail: str = ""):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}"
                         + (f" ({detail})" if detail else ""))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        how = ("`python -m paper_2209_14487_gb300.build --check`" if CHECKED else
               "`python -c 'import __graft_entry__ as g; g.build()'`")
        raise ImportError(f"{LIB_PATH} is missing: build it with {how} (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    vp, i = C.c_void_p, C.c_int
    sig = {
        "qmc_crowd_create": [C.POINTER(qmc_system_desc), C.POINTER(qmc_run_desc), vp,
                             C.POINTER(vp)],
        "qmc_crowd_destroy": [vp],
        "qmc_load_positions": [vp, vp, i],
        "qmc_load_ions": [vp, vp],
        "qmc_load_orbitals": [vp, vp, i, i],
        "qmc_load_jastrow": [vp, i, vp, i, C.c_double],
        "qmc_recompute": [vp],
        "qmc_eval_grad_batch": [vp, i, vp, i],
        "qmc_propose_move_batch": [vp, i, vp, vp, vp, vp, vp, i],
        "qmc_accept_reject_batch": [vp, i, vp, vp, i],
        "qmc_local_energy_batch": [vp, vp, i],
        "qmc_sweep": [vp, i, vp, i, C.POINTER(qmc_stats)],
        "qmc_get_positions": [vp, vp, i],
        "qmc_get_logpsi": [vp, vp, vp],
        "qmc_get_inverse": [vp, i, vp],
        "qmc_get_slater_matrix": [vp, i, vp],
        "qmc_get_generation": [vp, C.POINTER(C.c_uint32)],
        "qmc_set_generation": [vp, C.c_uint32],
        "qmc_get_launch_count": [vp, C.POINTER(C.c_ulonglong)],
        "qmc_get_kernel_config": [vp] + [C.POINTER(C.c_int)] * 6,
        "qmc_batch_create": [C.POINTER(vp), i, C.POINTER(vp)],
        "qmc_batch_destroy": [vp],
        "qmc_batch_sweep": [vp, i, vp, vp],
        "qmc_batch_get_launch_count": [vp, C.POINTER(C.c_ulonglong)],
        "qmc_dmc_branch": [vp, vp, vp, i, C.c_double, C.POINTER(qmc_dmc_stats)],
        "qmc_get_walker_count": [vp, C.POINTER(C.c_int)],
        "qmc_get_update": [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "qmc_get_guard": [vp, vp, C.POINTER(C.c_longlong)],
        "qmc_trace_accepts": [vp, i],
        "qmc_get_accept_trace": [vp, vp],
        "qmc_test_skip_stencil_copy": [vp, i],
        "qmc_check_report": [vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong)],
        "qmc_test_plant_bad_cell": [vp, i],
        "qmc_dmc_select": [vp, vp, i, i],
        "qmc_dmc_append": [vp, vp, i, i],
        "qmc_load_nlpp": [vp, i, vp, vp, C.c_double],
        "qmc_load_coulomb": [vp, i, C.c_double, C.c_double, i],
        "qmc_crowd_save": [vp, vp, C.POINTER(C.c_size_t)],
        "qmc_crowd_restore": [vp, vp, C.c_size_t],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.qmc_inverse_noalloc.argtypes = [vp, i, i, vp, vp, vp, vp]
    lib.qmc_inverse_noalloc.restype = C.c_int
    lib.qmc_last_cuda_error.argtypes = []
    lib.qmc_last_cuda_error.restype = C.c_char_p
    lib.qmc_status_string.argtypes = [C.c_int]
    lib.qmc_status_string.restype = C.c_char_p
    lib.qmc_build_flags.argtypes = []
    lib.qmc_build_flags.restype = C.c_int
    return lib


lib = _load()


def build_flags() -> int:
    """QMC_BUILD_CHECKED when the loaded library is the bounds-checked build, else 0."""
    return lib.qmc_build_flags()


def _check(fn: str, st: int):
    if st != QMC_OK:
        detail = lib.qmc_last_cuda_error().decode() if st == 3 else ""
        raise QmcError(fn, st, detail)


def _buf(x, dtype=np.float64):
    """(pointer, mem kind, keep-alive) of an array argument; None -> (None, None, None)."""
    if x is None:
        return None, None, None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype).name} array")
        return x.ctypes.data, QMC_MEM_HOST, x
    try:
        import torch
    except ImportError as e:  # pragma: no cover
        raise TypeError("expected a numpy array or a torch tensor") from e
    if isinstance(x, torch.Tensor):
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8,
               np.int32: torch.int32}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {tdt} tensor")
        return x.data_ptr(), (QMC_MEM_DEVICE if x.is_cuda else QMC_MEM_HOST), x
    raise TypeError("expected a numpy array or a torch tensor")


def _mem(*kinds) -> int:
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("all buffers of one call must be on the host or all on the device")
    return ks.pop() if ks else QMC_MEM_HOST


class Crowd:
    """One qmc_crowd handle; methods are the C calls with their arguments marshalled."""

    def __init__(self, n_up, n_dn, n_orb, n_ions, grid, L, n_walkers, tau, precision="fp64",
                 update="sm", delay_rank=1, n_recompute=0, drift=True, potential=True,
                 seed=14487, stream=None, staging="auto", cta_threads=0, engine="auto",
                 dmc=False, guard_tol=0.0, layout="auto"):
        self.sys = qmc_system_desc(n_up=n_up, n_dn=n_dn, n_orb=n_orb, n_ions=n_ions, grid=grid,
                                   reserved=0, L=L)
        self.run = qmc_run_desc(
            n_walkers=n_walkers,
            precision=QMC_PREC_MIXED if precision == "mixed" else QMC_PREC_FP64,
            update=QMC_UPDATE_DELAYED if update == "delayed" else QMC_UPDATE_SM,
            delay_rank=delay_rank, n_recompute=n_recompute, drift=int(drift),  # True: limited
            potential=int(potential), staging=QMC_STAGING_LDG if staging == "ldg" else QMC_STAGING_AUTO,
            tau=tau, seed=seed, cta_threads=cta_threads,
            engine=QMC_ENGINE_SIMT if engine == "simt" else QMC_ENGINE_AUTO,
            dmc=int(bool(dmc)), layout=LAYOUTS[layout], guard_tol=float(guard_tol))
        self.W, self.N, self.n = n_walkers, n_up + n_dn, n_up
        self.capacity = n_walkers
        h = C.c_void_p()
        _check("qmc_crowd_create",
               lib.qmc_crowd_create(C.byref(self.sys), C.byref(self.run), stream, C.byref(h)))
        self.h = h

    @classmethod
    def from_workload(cls, wl, precision="fp64", update="sm", delay_rank=1, n_walkers=None,
                      stream=None, n_recompute=None, staging="auto", cta_threads=0,
                      engine="auto", dmc=False, tau=None, guard_tol=0.0, layout="auto"):
        c = cls(wl.n_up, wl.n_dn, wl.n_orb, wl.n_ions, wl.grid, wl.L,
                wl.n_walkers if n_walkers is None else n_walkers,
                wl.tau if tau is None else tau, precision=precision,
                update=update, delay_rank=delay_rank,
                n_recompute=wl.n_recompute if n_recompute is None else n_recompute,
                drift=wl.drift, potential=wl.potential, seed=wl.seed, stream=stream,
                staging=staging, cta_threads=cta_threads, engine=engine, dmc=dmc,
                guard_tol=guard_tol, layout=layout)
        if wl.n_ions:
            c.qmc_load_ions(np.ascontiguousarray(wl.ions, dtype=np.float64))
        if wl.j2_uu is not None:
            c.qmc_load_jastrow(QMC_J2_UU, wl.j2_uu.coefs, wl.j2_uu.rc)
            c.qmc_load_jastrow(QMC_J2_UD, wl.j2_ud.coefs, wl.j2_ud.rc)
        if wl.j1 is not None:
            c.qmc_load_jastrow(QMC_J1, wl.j1.coefs, wl.j1.rc)
        c.qmc_load_orbitals(np.ascontiguousarray(wl.table(), dtype=np.float64))
        return c

    def close(self):
        if getattr(self, "h", None):
            lib.qmc_crowd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- inputs ----
    def qmc_load_positions(self, R):
        p, m, _ = _buf(R)
        _check("qmc_load_positions", lib.qmc_load_positions(self.h, p, m))

    def qmc_load_ions(self, RI):
        RI = np.ascontiguousarray(RI, dtype=np.float64)
        _check("qmc_load_ions", lib.qmc_load_ions(self.h, RI.ctypes.data))

    def qmc_load_orbitals(self, coefs):
        dt = np.float32 if getattr(coefs, "dtype", None) in (np.float32,) or \
            str(getattr(coefs, "dtype", "")) == "torch.float32" else np.float64
        p, m, _ = _buf(coefs, dt)
        _check("qmc_load_orbitals", lib.qmc_load_orbitals(
            self.h, p, QMC_DTYPE_F32 if dt == np.float32 else QMC_DTYPE_F64, m))

    def qmc_load_jastrow(self, kind, coefs, rc):
        c = np.ascontiguousarray(coefs, dtype=np.float64)
        _check("qmc_load_jastrow",
               lib.qmc_load_jastrow(self.h, kind, c.ctypes.data if c.size else None, c.size, rc))

    def qmc_recompute(self):
        _check("qmc_recompute", lib.qmc_recompute(self.h))

    # ---- the move ----
    def qmc_eval_grad_batch(self, iel, grad):
        p, m, _ = _buf(grad)
        _check("qmc_eval_grad_batch", lib.qmc_eval_grad_batch(self.h, iel, p, m))

    def qmc_propose_move_batch(self, iel, rnew=None, ratio=None, grad=None, log_ratio=None,
                               rnew_out=None):
        bs = [_buf(x) for x in (rnew, ratio, grad, log_ratio, rnew_out)]
        m = _mem(*[b[1] for b in bs])
        _check("qmc_propose_move_batch",
               lib.qmc_propose_move_batch(self.h, iel, *[b[0] for b in bs], m))

    def qmc_accept_reject_batch(self, iel, accept=None, accepted_out=None):
        a = _buf(accept, np.uint8)
        o = _buf(accepted_out, np.uint8)
        m = _mem(a[1], o[1])
        _check("qmc_accept_reject_batch", lib.qmc_accept_reject_batch(self.h, iel, a[0], o[0], m))

    def qmc_local_energy_batch(self, eloc):
        p, m, _ = _buf(eloc)
        _check("qmc_local_energy_batch", lib.qmc_local_energy_batch(self.h, p, m))

    def qmc_sweep(self, n_gen, eloc=None, stats=True):
        p, m, _ = _buf(eloc)
        st = qmc_stats() if stats else None
        _check("qmc_sweep", lib.qmc_sweep(self.h, n_gen, p, m if m is not None else 0,
                                          C.byref(st) if st is not None else None))
        return st

    # ---- getters ----
    def qmc_get_positions(self, R=None):
        if R is None:
            R = np.zeros((self.W, self.N, 3))
        p, m, _ = _buf(R)
        _check("qmc_get_positions", lib.qmc_get_positions(self.h, p, m))
        return R

    def qmc_get_logpsi(self):
        la = np.zeros(self.W)
        sg = np.zeros(self.W, dtype=np.int32)
        _check("qmc_get_logpsi", lib.qmc_get_logpsi(self.h, la.ctypes.data, sg.ctypes.data))
        return la, sg

    def qmc_get_inverse(self, spin):
        out = np.zeros((self.W, self.n, self.n))
        _check("qmc_get_inverse", lib.qmc_get_inverse(self.h, spin, out.ctypes.data))
        return out

    def qmc_get_slater_matrix(self, spin):
        out = np.zeros((self.W, self.n, self.n))
        _check("qmc_get_slater_matrix", lib.qmc_get_slater_matrix(self.h, spin, out.ctypes.data))
        return out

    @property
    def generation(self) -> int:
        g = C.c_uint32()
        _check("qmc_get_generation", lib.qmc_get_generation(self.h, C.byref(g)))
        return g.value

    @generation.setter
    def generation(self, g: int):
        _check("qmc_set_generation", lib.qmc_set_generation(self.h, g))

    @property
    def launch_count(self) -> int:
        v = C.c_ulonglong()
        _check("qmc_get_launch_count", lib.qmc_get_launch_count(self.h, C.byref(v)))
        return v.value

    @property
    def kernel_config(self) -> dict:
        """{'b_in_smem', 'stencil_tma', 'smem_bytes', 'cta_threads', 'tc_flush', 'layout'}
        of the move kernel (layout: 'shared' or 'compact')."""
        v = [C.c_int() for _ in range(6)]
        _check("qmc_get_kernel_config",
               lib.qmc_get_kernel_config(self.h, *[C.byref(x) for x in v]))
        d = dict(zip(("b_in_smem", "stencil_tma", "smem_bytes", "cta_threads", "tc_flush"),
                     (x.value for x in v[:5])))
        d["layout"] = "compact" if v[5].value == QMC_LAYOUT_COMPACT else "shared"
        return d

    def qmc_dmc_branch(self, e_prev, e_new, e_trial: float):
        """DMC reweighting and branching after a generation (host arrays [W]); returns
        (qmc_dmc_stats, E_L of the new population).  The crowd's walker count changes."""
        ep = np.ascontiguousarray(e_prev, dtype=np.float64)
        # the gathered E_L of the new population, up to the capacity
        en = np.zeros(self.capacity, dtype=np.float64)
        en[:len(e_new)] = e_new
        st = qmc_dmc_stats()
        _check("qmc_dmc_branch", lib.qmc_dmc_branch(self.h, ep.ctypes.data, en.ctypes.data,
                                                    QMC_MEM_HOST, float(e_trial),
                                                    C.byref(st)))
        self.W = st.n_after
        return st, en[:st.n_after].copy()

    def qmc_load_nlpp(self, amps, widths, rc):
        """Nonlocal channels l = 0..len(amps)-1 in every E_L from now on (empty: none)."""
        a = np.ascontiguousarray(amps, dtype=np.float64)
        w = np.ascontiguousarray(widths, dtype=np.float64)
        if a.shape != w.shape:
            raise ValueError("one width per amplitude")
        _check("qmc_load_nlpp", lib.qmc_load_nlpp(self.h, int(a.size), a.ctypes.data,
                                                  w.ctypes.data, float(rc)))

    def qmc_load_coulomb(self, Z, alpha, mmax, on=True):
        """Ewald Coulomb energy (electrons -1, ions +Z) in every E_L from now on."""
        _check("qmc_load_coulomb", lib.qmc_load_coulomb(self.h, int(bool(on)), float(Z),
                                                        float(alpha), int(mmax)))

    def qmc_dmc_select(self, src):
        """The new population is walkers src (indices into the current one, in order)."""
        if not hasattr(src, "data_ptr"):  # anything but a torch tensor: a host int32 copy
            src = np.ascontiguousarray(src, dtype=np.int32)
        p, m, keep = _buf(src, np.int32)
        n_new = int(keep.shape[0])
        _check("qmc_dmc_select", lib.qmc_dmc_select(self.h, p, n_new, m))
        self.W = n_new

    def qmc_dmc_append(self, R):
        """Walkers with positions R [m][N][3] join the crowd (their inverses are built)."""
        p, m, keep = _buf(R)
        n_add = int(keep.shape[0])
        _check("qmc_dmc_append", lib.qmc_dmc_append(self.h, p, n_add, m))
        self.W += n_add

    @property
    def delay_rank(self) -> int:
        """The delay rank in use (the library's pick when created with delay_rank=0)."""
        u, k = C.c_int(), C.c_int()
        _check("qmc_get_update", lib.qmc_get_update(self.h, C.byref(u), C.byref(k)))
        return k.value

    def qmc_get_guard(self):
        """(probe value of every walker's last sweep [W], repairs since creation)."""
        v = np.zeros(self.W)
        nr = C.c_longlong()
        _check("qmc_get_guard", lib.qmc_get_guard(self.h, v.ctypes.data, C.byref(nr)))
        return v, nr.value

    def qmc_trace_accepts(self, on: bool = True):
        _check("qmc_trace_accepts", lib.qmc_trace_accepts(self.h, int(bool(on))))

    def qmc_get_accept_trace(self):
        """Accept decisions [W][N] (uint8) of the last generation swept while recording."""
        out = np.zeros((self.W, self.N), dtype=np.uint8)
        _check("qmc_get_accept_trace", lib.qmc_get_accept_trace(self.h, out.ctypes.data))
        return out

    def qmc_test_skip_stencil_copy(self, on: bool):
        """Failure-detection test hook: stencil copies not issued (their waits run out)."""
        _check("qmc_test_skip_stencil_copy",
               lib.qmc_test_skip_stencil_copy(self.h, int(bool(on))))

    def qmc_check_report(self):
        """(site, value) of the crowd's first failed bounds check since the last report
        (site 0: none; always 0 outside the bounds-checked build)."""
        site, val = C.c_int(), C.c_longlong()
        _check("qmc_check_report", lib.qmc_check_report(self.h, C.byref(site), C.byref(val)))
        return site.value, val.value

    def qmc_test_plant_bad_cell(self, on: bool):
        """Checked-build test hook: electron 0's proposals get an out-of-range cell."""
        _check("qmc_test_plant_bad_cell", lib.qmc_test_plant_bad_cell(self.h, int(bool(on))))

    @property
    def walker_count(self) -> int:
        v = C.c_int()
        _check("qmc_get_walker_count", lib.qmc_get_walker_count(self.h, C.byref(v)))
        return v.value

    def qmc_crowd_save(self) -> bytes:
        sz = C.c_size_t()
        _check("qmc_crowd_save", lib.qmc_crowd_save(self.h, None, C.byref(sz)))
        buf = C.create_string_buffer(sz.value)
        _check("qmc_crowd_save", lib.qmc_crowd_save(self.h, buf, C.byref(sz)))
        return buf.raw[:sz.value]

    def qmc_crowd_restore(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _check("qmc_crowd_restore", lib.qmc_crowd_restore(self.h, buf, len(data)))


class Batch:
    """Crowds of different systems swept together: one launch per generation covers every
    walker of every crowd (qmc_batch_* in include/qmcgb.h).  Keeps the crowds alive."""

    def __init__(self, crowds):
        self.crowds = list(crowds)
        arr = (C.c_void_p * len(self.crowds))(*[c.h.value for c in self.crowds])
        h = C.c_void_p()
        _check("qmc_batch_create", lib.qmc_batch_create(arr, len(self.crowds), C.byref(h)))
        self.h = h

    def qmc_batch_sweep(self, n_gen: int, eloc=True, stats=True):
        """(list of E_L arrays [n_gen][W_c] or None, list of qmc_stats or None)."""
        out = [np.zeros((n_gen, c.W)) for c in self.crowds] if eloc else None
        ptrs = (C.c_void_p * len(self.crowds))(*[o.ctypes.data for o in out]) if eloc else None
        st = (qmc_stats * len(self.crowds))() if stats else None
        _check("qmc_batch_sweep", lib.qmc_batch_sweep(self.h, n_gen, ptrs, st))
        return out, (list(st) if stats else None)

    @property
    def launch_count(self) -> int:
        v = C.c_ulonglong()
        _check("qmc_batch_get_launch_count", lib.qmc_batch_get_launch_count(self.h, C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None):
            lib.qmc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qmc_inverse_noalloc(a, inv, logdet, sign, stream=None):
    """FP64 inverse, log|det| and sign of a batch of n x n matrices without any device
    allocation (all four arguments are CUDA tensors: a, inv float64 [batch][n][n], logdet
    float64 [batch], sign int32 [batch]); asynchronous on `stream` (a cudaStream_t
    handle, None for the legacy default stream)."""
    import torch
    for t in (a, inv, logdet, sign):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise TypeError("qmc_inverse_noalloc takes contiguous CUDA tensors")
    if a.dtype != torch.float64 or inv.dtype != torch.float64 or logdet.dtype != torch.float64 \
            or sign.dtype != torch.int32:
        raise TypeError("a, inv, logdet: float64; sign: int32")
    batch, n = a.shape[0], a.shape[-1]
    _check("qmc_inverse_noalloc", lib.qmc_inverse_noalloc(
        a.data_ptr(), n, batch, inv.data_ptr(), logdet.data_ptr(), sign.data_ptr(), stream))


def qmc_status_string(st: int) -> str:
    return lib.qmc_status_string(st).decode()
