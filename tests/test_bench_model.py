"""The benchmark's per-move byte model (the roofline numerator) against the worked
examples of the scope table's measurement section, at acceptance 0.5."""
import pytest

import bench


@pytest.mark.parametrize("n,N,s,update,k,expect", [
    (256, 512, 8, "sm", 1, 0.695e6),         # C3 FP64 Sherman-Morrison: ~0.70 MB per move
    (256, 512, 4, "delayed", 16, 0.144e6),   # C3 mixed, k = 16: ~144 KB
    (768, 1536, 4, "delayed", 32, 0.567e6),  # C5 mixed, k = 32: ~567 KB
])
def test_bytes_per_move_examples(n, N, s, update, k, expect):
    b = bench.bytes_per_move(n, N, s, 0.5, update, k)
    assert abs(b - expect) < 0.02 * expect, b


def test_aggregate_value_single_rank():
    assert bench.aggregate_value(1000.0, 2.0, 1) == 500.0
    assert bench.reduce_sum(3.5, 1) == 3.5


def test_amortised_recompute_share():
    """A step without the recompute gets (recompute generation - plain generation) /
    n_recompute added; a step that carried one keeps its own time."""
    r = {"ms": [1.0, 1.0, 5.0, 1.0], "plain_ms": [1.0, 1.0, 1.0], "due": [False, False, True, False],
         "recompute_step_ms": [9.0, 9.0]}
    ms, extra = bench.amortised(r, 4)
    assert extra == pytest.approx(8.0)
    assert ms == pytest.approx([3.0, 3.0, 5.0, 3.0])
    assert bench.amortised(dict(r, recompute_step_ms=[]), 4) == (r["ms"], 0.0)
    assert bench.amortised(r, 0) == (r["ms"], 0.0)


def test_energy_stats_blocks():
    """Block means of the crowd average per generation: the mean of all generations and the
    standard error of the block means; fewer than two blocks give no error."""
    np = pytest.importorskip("numpy")
    e = np.repeat(np.arange(8.0)[:, None], 3, axis=1)  # generation g: every walker g
    m, s = bench.energy_stats(e, block=2)
    b = np.array([0.5, 2.5, 4.5, 6.5])
    assert m == pytest.approx(b.mean())
    assert s == pytest.approx(b.std(ddof=1) / 2.0)
    m1, s1 = bench.energy_stats(e, block=8)
    assert m1 == pytest.approx(3.5) and s1 != s1  # NaN
