"""The seeded generator against a scalar restatement of SplitMix64's published
definition (Steele, Lea, Flood, OOPSLA 2014) in Python integers."""
import numpy as np

from paper_2306_11686_gb300 import inputs

MASK = (1 << 64) - 1


def splitmix_scalar(seed, k):
    z = (seed * 0x9E3779B97F4A7C15 + (k + 1) * 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_splitmix_counter_form():
    v = inputs.splitmix64(12345, 50, offset=3)
    assert [int(a) for a in v] == [splitmix_scalar(12345, k) for k in range(3, 53)]


def test_sequential_generator_equivalence():
    # the counter form equals the sequential generator with state seed*GOLDEN
    state = (99 * 0x9E3779B97F4A7C15) & MASK
    out = []
    for _ in range(10):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    assert [int(a) for a in inputs.splitmix64(99, 10)] == out


def test_uniform_ranges_exact():
    u = inputs.uniform_pm1(5, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0
    # 2u-1 is exact: u recovers bit-for-bit
    assert np.array_equal((u + 1.0) / 2.0, inputs.uniform01(5, 100000))


def test_loguniform_per_octave():
    v = inputs.loguniform_int(3, 200000, 16, 65536)
    assert v.min() >= 16 and v.max() <= 65536
    octs = np.bincount(np.floor(np.log2(v)).astype(int))[4:16]
    assert octs.min() > 0.8 * octs.mean()


def test_jacobi_input_boundary():
    g = inputs.jacobi_input(10, 2).reshape(10, 10, 10)
    assert not g[0].any() and not g[:, :, -1].any()
    assert g[1:-1, 1:-1, 1:-1].min() >= 0.0 and g.max() < 1.0
