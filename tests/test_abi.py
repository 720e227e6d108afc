"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/qmcgb.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qmcgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qmc_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2209_14487_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2209_14487_gb300 import qmcgb
    assert sorted(qmcgb.EXPORTS) == names


def test_status_strings_without_gpu():
    from paper_2209_14487_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.qmc_status_string.restype = ctypes.c_char_p
    assert lib.qmc_status_string(0) == b"ok"
    assert b"singular" in lib.qmc_status_string(4)
    assert lib.qmc_status_string(99) == b"unknown status"


def test_invalid_arguments_rejected_before_device_use():
    from paper_2209_14487_gb300 import qmcgb
    Q = qmcgb
    h = ctypes.c_void_p()
    sys_ = Q.qmc_system_desc(n_up=4, n_dn=4, n_orb=4, n_ions=0, grid=8, reserved=0, L=3.0)
    run = Q.qmc_run_desc(n_walkers=0, precision=0, update=0, delay_rank=1, n_recompute=0,
                         drift=1, potential=1, staging=0, tau=0.3, seed=1,
                         cta_threads=0, engine=0, dmc=0, layout=0)
    assert Q.lib.qmc_crowd_create(ctypes.byref(sys_), ctypes.byref(run), None,
                                  ctypes.byref(h)) == 1
    run.n_walkers = 2
    run.update = 1
    run.delay_rank = 65
    assert Q.lib.qmc_crowd_create(ctypes.byref(sys_), ctypes.byref(run), None,
                                  ctypes.byref(h)) == 1
    run.update = 0
    sys_.n_dn = 3  # open shell: not served by this build
    assert Q.lib.qmc_crowd_create(ctypes.byref(sys_), ctypes.byref(run), None,
                                  ctypes.byref(h)) == 8
    assert Q.lib.qmc_crowd_destroy(None) == 1


def _enum_values(prefix):
    src = open(os.path.join(ROOT, "include", "qmcgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {m.group(1): int(m.group(2))
            for m in re.finditer(r"\b(" + prefix + r"[A-Z0-9_]*)\s*=\s*(\d+)", src)}


def test_binding_constants_match_the_header():
    """Every status, layout and build-flag constant the binding uses has the header's
    value, and every status code has its name and its text."""
    from paper_2209_14487_gb300 import build, qmcgb
    errs = _enum_values("QMC_ERR_")
    errs["QMC_OK"] = _enum_values("QMC_OK")["QMC_OK"]
    assert qmcgb.STATUS_NAMES == {v: k for k, v in errs.items()}
    layouts = _enum_values("QMC_LAYOUT_")
    assert (qmcgb.QMC_LAYOUT_AUTO, qmcgb.QMC_LAYOUT_SHARED, qmcgb.QMC_LAYOUT_COMPACT) == (
        layouts["QMC_LAYOUT_AUTO"], layouts["QMC_LAYOUT_SHARED"], layouts["QMC_LAYOUT_COMPACT"])
    assert qmcgb.QMC_BUILD_CHECKED == _enum_values("QMC_BUILD_")["QMC_BUILD_CHECKED"]
    assert qmcgb.QMC_ERR_BOUNDS == errs["QMC_ERR_BOUNDS"]
    lib = ctypes.CDLL(build.build())
    lib.qmc_status_string.restype = ctypes.c_char_p
    for code in errs.values():
        assert lib.qmc_status_string(code) != b"unknown status", code
    lib.qmc_build_flags.restype = ctypes.c_int
    assert lib.qmc_build_flags() == 0  # the normal build
