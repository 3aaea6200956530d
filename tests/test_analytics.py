"""DRX analytics (post-processing of coupled-run statistics) against constructed cases."""
import math

import numpy as np

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
