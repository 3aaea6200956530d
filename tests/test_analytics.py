"""DRX analytics (post-processing of coupled-run statistics) against constructed cases."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1509_04953_gb300 import analytics as A
from paper_1509_04953_gb300 import synth


def test_avrami_fit_recovers_exponent_and_rate():
    t = np.linspace(0, 50, 200)
    t0, m, K = 5.0, 1.42, 3e-3
    X = np.where(t > t0, 1 - np.exp(-K * np.clip(t - t0, 0, None) ** m), 0.0)
    mm, KK = A.avrami_fit(t, X, t0=t0)
    assert abs(mm - m) < 1e-9 and abs(KK / K - 1) < 1e-8


def test_critical_strain_is_first_nucleation():
    assert A.critical_strain([0.01, 0.02, 0.03, 0.04], [0, 0, 3, 1]) == 0.03
    assert A.critical_strain([0.01, 0.02], [0, 0]) is None


def test_expected_nuclei_matches_the_oracle_nucleation_statistics(mat):
    """The expected count from the k field equals the mean number of nuclei the (oracle) Weibull
    nucleation produces on fresh strengths, within sampling error."""
    n, G = 16, 6
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, 2))
    k = np.random.default_rng(0).uniform(0.3, 0.9, n ** 3) * mat.kc
    want = A.expected_nuclei(k, g0, n, mat.kc, mat.q)
    counts = []
    for seed in range(12):
        st = O.State(n, G, g0, synth.orientations(G, 2), mat, seed=100 + seed)
        st.field("k")[0, :] = k
        counts.append(st.nucleate(0)[1])
    mean, sd = np.mean(counts), np.std(counts) / math.sqrt(len(counts))
    assert abs(mean - want) < 5 * sd + 1.0


def test_grain_statistics():
    g = np.repeat(np.arange(8), 64)
    ng, d = A.grain_statistics(g, 8, dx=2.0)
    assert ng == 8 and abs(d - (6 * 64 * 8 / math.pi) ** (1 / 3)) < 1e-12


def _flood_fill_count(g, n):
    """Brute force: count 6-connected periodic same-id components by breadth-first search."""
    g = np.asarray(g).reshape(n, n, n)
    seen = np.zeros_like(g, dtype=bool)
    count = 0
    for start in np.ndindex(n, n, n):
        if seen[start]:
            continue
        count += 1
        stack = [start]
        seen[start] = True
        while stack:
            z, y, x = stack.pop()
            for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                w = ((z + dz) % n, (y + dy) % n, (x + dx) % n)
                if not seen[w] and g[w] == g[z, y, x]:
                    seen[w] = True
                    stack.append(w)
    return count


def test_grain_components_are_periodic_six_neighbour_regions():
    n = 8
    g = np.zeros((n, n, n), dtype=np.int32)
    g[:, :, 0:2] = 1          # a slab at x = 0, 1 ...
    g[:, :, 7] = 1            # ... continues across the periodic wrap: one grain
    g[2:4, 2:4, 4:6] = 2      # two separate blocks of id 2: two grains
    g[5:7, 5:7, 4:6] = 2
    g[0, 4, 3] = 3            # id 3 at two voxels touching only along an edge: two grains (6-neighbour)
    g[1, 5, 3] = 3
    ng, labels = A.grain_components(g.reshape(-1), n)
    assert ng == 1 + 1 + 2 + 2              # id 0 (the rest, one region), slab, two blocks, two single voxels
    assert ng == _flood_fill_count(g, n)
    lab = labels.reshape(n, n, n)
    assert lab[0, 0, 0] == lab[0, 0, 7] and lab[2, 2, 4] != lab[5, 5, 4] and lab[0, 4, 3] != lab[1, 5, 3]


def test_grain_components_match_brute_force_on_random_voronoi():
    for seed, (n, G) in enumerate([(6, 5), (8, 12), (10, 30)]):
        g = O.voronoi(n, synth.voronoi_seeds(n, G, 40 + seed))
        rng = np.random.default_rng(seed)
        g = np.where(rng.random(g.size) < 0.1, G + rng.integers(0, 3, g.size), g)   # scattered "nuclei"
        assert A.grain_components(g, n)[0] == _flood_fill_count(g, n)


def test_grain_statistics_mean_equivalent_diameter():
    n = 4
    g = np.zeros((n, n, n), dtype=np.int32)
    g[:, :, 2:] = 1                          # two grains of 32 voxels
    g[0, 0, 0] = 2                           # and one of 1 voxel
    ng, d = A.grain_statistics(g.reshape(-1), n, dx=0.5)
    vols = np.array([31.0, 32.0, 1.0]) * 0.125
    assert ng == 3 and d == pytest.approx(np.mean((6 * vols / math.pi) ** (1 / 3)), rel=1e-14)
