"""The seeded input generator against the published SplitMix64 definition."""
import numpy as np

from synth import splitmix64, uniform_pm1


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0: the first outputs of the reference generator
    # (Steele, Lea, Flood 2014; the seeding routine of the xoshiro family).
    z = splitmix64(0, np.arange(2, dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_uniform_range_and_determinism():
    a = uniform_pm1(100000, 3)
    b = uniform_pm1(100000, 3)
    c = uniform_pm1(100000, 4)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0 / 3.0) < 0.01
    assert uniform_pm1(0, 1).size == 0


def test_batched_and_served_workloads_follow_their_recipes():
    """The batched mix and the served problems of the bench (no GPU): sizes 2^10..2^18 (batch)
    and 2^10..2^22 (serving) unknowns, r = floor(delta 2^K) >= 1, the kernel and transfer rules."""
    import bench
    specs = bench.batch_mix_workload(512)
    assert len(specs) == 512 and specs == bench.batch_mix_workload(512)   # seeded
    n2 = 0
    for dim, K, delta, v, kk, a in specs:
        n = ((1 << (K + 1)) - 1) ** dim
        assert 2 ** 9 < n < 2 ** 18 + 1 and 0.02 <= delta <= 0.25 and delta * (1 << K) >= 1.0
        if dim == 2:
            n2 += 1
            assert kk == 0 and 4 <= K <= 8
        elif kk:
            assert v == 0 and 0.1 <= a <= 0.4 and 9 <= K <= 17
    assert 0 < n2 < 512
    one, two = bench.serve_keys()
    for dim, v, d, K, kk, a, tr in one + two:
        n = ((1 << (K + 1)) - 1) ** dim
        assert 2 ** 9 < n < 2 ** 22 + 1 and d * (1 << K) >= 1.0
        assert (kk == 1) == (tr == 1) and (kk == 0 or (v == 0 and a <= 0.4))
    assert {k[0] for k in two} == {2} and {k[0] for k in one} == {1}
