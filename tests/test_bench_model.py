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
