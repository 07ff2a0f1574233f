"""The batched-workload shapes (synth.batched_workload): deterministic in the seeds, inside the stated
ranges, t = n, and roughly uniform over them (a simple count check over many circuits)."""
from synth import batched_workload


def test_shapes_are_deterministic_and_in_range():
    a = batched_workload(256)
    assert a == batched_workload(256)
    assert [x[3] for x in a] == list(range(256))
    for n, layers, t, _seed in a:
        assert 16 <= n <= 48 and 16 <= layers <= 48 and t == n
    b = batched_workload(8, seed0=1000, n_range=(16, 24), layer_range=(16, 24))
    assert all(16 <= n <= 24 and 16 <= layers <= 24 for n, layers, _t, _s in b)
    assert batched_workload(4, seed0=256) == batched_workload(260)[256:]


def test_shapes_cover_the_range():
    a = batched_workload(4000, n_range=(16, 19), layer_range=(16, 19))
    for k in (0, 1):
        counts = [sum(1 for x in a if x[k] == v) for v in range(16, 20)]
        assert min(counts) > 850 and max(counts) < 1150      # 1000 expected per value
