"""The bounds-checked build (the same sources with -DQMCGB_CHECK=1, libqmcgb_check.so) runs
a cross-section of the oracle parity tests in a child process with QMCGB_CHECK=1: the
smallest systems and the planted bad cell, the FP64 trajectories at three CTA widths, the
mixed ratios with the TMA-staged stencil, the incremental Jastrow, the inverse guard's
repair, the DMC branch and gather, the nonlocal pair list and the batch kernel.  A device
check that fires makes its call return QMC_ERR_BOUNDS, so the child's tests fail; they
must all pass."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SUBSET = [
    "tests/test_gpu_small_systems.py",
    "tests/test_gpu_parity.py::test_fp64_propose_accept_sequence",
    "tests/test_gpu_parity.py::test_fp64_delayed_update_matches_oracle",
    "tests/test_gpu_parity.py::test_fp64_sweep_trajectory_matches_oracle",
    "tests/test_gpu_parity.py::test_edge_cases_and_errors",
    "tests/test_gpu_parity.py::test_mixed_ratios_within_tolerance",
    "tests/test_gpu_parity.py::test_incremental_jastrow_matches_full_pass",
    "tests/test_gpu_guard.py::test_guard_repair_equals_fp64_recompute",
    "tests/test_gpu_dmc.py",
    "tests/test_gpu_nlpp.py",
    "tests/test_gpu_batch.py",
]


def test_checked_build_passes_parity_subset():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_14487_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, QMCGB_CHECK="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           *SUBSET]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout[-4000:] + "\n" + r.stderr[-2000:]).strip()
    print(tail)
    assert r.returncode == 0 and " passed" in r.stdout, tail
