"""The autotuner's host logic without a GPU: the candidate table, the fastest pick, the
per-GPU cache, and the plan stage that times each distinct kernel plan once.  The crowd
and the timing call are replaced by fakes (the timing itself needs a GB300)."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2209_14487_gb300 import autotune  # noqa: E402
from paper_2209_14487_gb300 import workloads as wl_mod  # noqa: E402


class FakeCrowd:
    """kernel_config of a crowd built with (staging, layout): the library folds the
    requested layout 'shared' and 'compact' into the same plan for this fake system when
    fold_layout is set (as it does where compact brings nothing)."""

    fold_layout = False

    def __init__(self, staging, layout):
        lay = "shared" if (self.fold_layout or layout == "auto") else layout
        self.kernel_config = {"stencil_tma": 0 if staging == "ldg" else 1, "layout": lay,
                              "b_in_smem": 1, "tc_flush": 0}

    @classmethod
    def from_workload(cls, wl, **kw):
        return cls(kw.get("staging", "auto"), kw.get("layout", "auto"))

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch, tmp_path):
    qmcgb = pytest.importorskip("paper_2209_14487_gb300.qmcgb")  # the built library
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    monkeypatch.setenv("QMCGB_TUNE_CACHE", str(tmp_path / "cache.json"))
    monkeypatch.setattr(qmcgb, "Crowd", FakeCrowd)
    calls = []

    def time_candidate(wl, precision, update, k, gens=4, warmup=2, cta_threads=0,
                       staging="auto", layout="auto", want=None):
        calls.append((update, k, cta_threads, staging, layout))
        ms = {("sm", 1): 3.0, ("delayed", 8): 2.0, ("delayed", 16): 2.5}[(update, k)]
        ms += {128: 0.0, 256: 0.5}[cta_threads]
        ms += {"auto": 0.0, "ldg": 0.3}[staging] + {"auto": 0.0, "shared": 0.0,
                                                     "compact": 0.2}[layout]
        return ms

    monkeypatch.setattr(autotune, "time_candidate", time_candidate)
    FakeCrowd.fold_layout = False
    return calls, tmp_path / "cache.json"


def test_tune_picks_the_fastest_and_caches(fake):
    calls, cache = fake
    wl = wl_mod.pw16()
    cands = (("sm", 1), ("delayed", 8), ("delayed", 16))
    update, k, nt, table = autotune.tune(wl, "mixed", candidates=cands, widths=(128, 256))
    assert (update, k, nt) == ("delayed", 8, 128)
    assert set(table) == {f"{u}:{kk}:{w}" for u, kk in cands for w in (128, 256)}
    assert len(calls) == 6
    entry = json.load(open(cache))
    assert any(e["update"] == "delayed" and e["k"] == 8 for e in entry.values())
    # a second call is served from the cache: no timing
    assert autotune.tune(wl, "mixed", candidates=cands, widths=(128, 256))[:3] == (update, k, nt)
    assert len(calls) == 6


def test_tune_plan_times_each_distinct_plan_once(fake):
    calls, _ = fake
    wl = wl_mod.pw16()
    staging, layout, table = autotune.tune_plan(wl, "mixed", "delayed", 8, 128)
    assert (staging, layout) == ("auto", "shared")
    assert set(table) == {"auto:shared", "auto:compact", "ldg:shared", "ldg:compact"}
    assert table["ldg:compact"] == pytest.approx(2.0 + 0.3 + 0.2)
    # where the library builds compact as shared, the duplicate plans are not timed
    FakeCrowd.fold_layout = True
    n0 = len(calls)
    _, _, table2 = autotune.tune_plan(wl, "fp64", "delayed", 8, 128)
    assert set(table2) == {"auto:shared", "ldg:shared"}
    assert len(calls) - n0 == 2
