"""The seeded input generator matches its published definition (CPU only)."""
import numpy as np

from paper_2101_12149_gb300 import inputs

M64 = (1 << 64) - 1


def _splitmix64(x):
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_reference_sequence():
    """SplitMix64 from state 1234567: the reference implementation's first outputs."""
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    got = [_splitmix64((1234567 + i * 0x9E3779B97F4A7C15) & M64) for i in range(5)]
    assert got == ref


def test_uniform_matches_definition():
    seed = 42
    key = _splitmix64(seed)
    u = inputs.uniform(seed, 100, 50, 3)
    for t in range(50):
        c = (100 + t) * 16 + 3
        ref = (_splitmix64((key + c) & M64) >> 11) * 2.0 ** -53
        assert u[t] == ref


def test_plasma_layout_and_ranges():
    n = (4, 3, 5)
    p = inputs.uniform_plasma(7, n, 3, sigma_u=0.1, density=2.0)
    N = 4 * 3 * 5 * 3
    assert all(p[k].size == N for k in p)
    cell = np.repeat(np.arange(60), 3)
    i, j, k = cell // 15, (cell // 5) % 3, cell % 5
    assert np.all((p["x"] >= i) & (p["x"] < i + 1))
    assert np.all((p["y"] >= j) & (p["y"] < j + 1))
    assert np.all((p["z"] >= k) & (p["z"] < k + 1))
    assert np.allclose(p["w"], 2.0 / 3)
    # sub-range generation reproduces the same particles
    q = inputs.uniform_plasma(7, n, 3, sigma_u=0.1, density=2.0, cells=(10, 20))
    for key in p:
        assert np.array_equal(q[key], p[key][30:60])


def test_normal_moments():
    z = inputs.normal(5, 0, 200000, 3)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
