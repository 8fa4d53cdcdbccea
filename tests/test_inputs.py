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


def test_ensemble_boxes_follow_the_recipe():
    boxes = inputs.ensemble_boxes()
    assert len(boxes) == 96
    edges = set(inputs.ENSEMBLE["edges"])
    for b in boxes:
        assert set(b["n"]) <= edges
        assert 1 <= b["ppc"] <= 8
        assert 0.1 <= b["density"] <= 10.0
        assert b["order"] in (1, 3)
    # every edge, particle count and both orders occur; seeds are distinct
    assert {e for b in boxes for e in b["n"]} == edges
    assert {b["ppc"] for b in boxes} == set(range(1, 9))
    assert len({b["seed"] for b in boxes}) == 96
    # log-uniform densities: about half below the geometric mean 1
    below = sum(b["density"] < 1.0 for b in boxes)
    assert 30 <= below <= 66
    # the same seed gives the same boxes
    assert inputs.ensemble_boxes() == boxes


def test_ensemble_particles_concatenate_in_box_order():
    boxes = inputs.ensemble_boxes(nboxes=4, edges=(8, 16))
    cat, counts, parts = inputs.ensemble_particles(boxes)
    assert counts.tolist() == [int(np.prod(b["n"])) * b["ppc"] for b in boxes]
    off = np.concatenate([[0], np.cumsum(counts)])
    for i, p in enumerate(parts):
        assert np.array_equal(cat["x"][off[i]:off[i + 1]], p["x"])
        assert np.allclose(p["w"], boxes[i]["density"] / boxes[i]["ppc"])
