"""DRX analytics on the per-increment statistics of a coupled run (post-processing, host side).

The paper analyses its coupled runs by the critical strain of the first nucleation event (Sec. 3,
Table CriticalStrainDRX), the expected number of nuclei as the overlap of the propensity
distribution f(k) with the strength density f_kappa(k) (Sec. 3, following Eq. NuclStrengthProb), the
recrystallised fraction with its Avrami exponent (Eq. Avrami) and the grain count and mean grain size
(Fig. Statistics). These functions compute the same quantities from what the library reports:
nuclei per increment (drx_nucleate), X_rex and n_grains (pf_step), and the k and grain-id fields.
"""
from __future__ import annotations

import math

import numpy as np


def critical_strain(strain, nuclei):
    """Macroscopic strain of the first increment that created a nucleus (None if none did)."""
    for e, n in zip(strain, nuclei):
        if n > 0:
            return float(e)
    return None


def boundary_mask(grain_id, n):
    """Voxels with a face neighbour of another grain (periodic), the nucleation sites."""
    g = np.asarray(grain_id).reshape(n, n, n)
    m = np.zeros_like(g, dtype=bool)
    for ax in range(3):
        for sh in (1, -1):
            m |= g != np.roll(g, sh, axis=ax)
    return m.reshape(-1)


def expected_nuclei(k, grain_id, n, kc, q):
    """Expected number of nuclei if every boundary voxel drew a fresh strength now:
    sum over boundary voxels of P(kappa < k) = 1 - exp(-(k/kc)^q) (Eq. NumCrt); the discrete form of
    the overlap integral of the propensity histogram with the strength density."""
    kk = np.asarray(k, dtype=np.float64).reshape(-1)[boundary_mask(grain_id, n)]
    return float(np.sum(1.0 - np.exp(-(kk / kc) ** q)))


def avrami_fit(t, X, x_lo=0.05, x_hi=0.95, t0=None):
    """Fit X = 1 - exp(-K (t - t0)^m) over x_lo < X < x_hi (Eq. Avrami): least squares of
    ln(-ln(1-X)) against ln(t - t0). t0 defaults to the last time with X = 0. Returns (m, K)."""
    t = np.asarray(t, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    if t0 is None:
        zero = np.nonzero(X <= 0.0)[0]
        t0 = float(t[zero[-1]]) if len(zero) else 0.0
    sel = (X > x_lo) & (X < x_hi) & (t > t0)
    if sel.sum() < 2:
        raise ValueError("not enough points inside the fitting window")
    yv = np.log(-np.log(1.0 - X[sel]))
    xv = np.log(t[sel] - t0)
    m, c = np.polyfit(xv, yv, 1)
    return float(m), float(math.exp(c))


def grain_components(grain_id, n):
    """Label grains as connected components: two voxels belong to the same grain when a chain of face
    neighbours (6-neighbour, periodic) with their grain id joins them. One id can form several grains (a
    recrystallised id that two growth fronts split, a deformed grain cut by a new one). Returns
    (number of grains, label per voxel in 0..number-1)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    g = np.asarray(grain_id).reshape(n, n, n)
    N3 = g.size
    idx = np.arange(N3, dtype=np.int64).reshape(n, n, n)
    rows, cols = [], []
    for ax in range(3):
        same = g == np.roll(g, -1, axis=ax)
        rows.append(idx[same])
        cols.append(np.roll(idx, -1, axis=ax)[same])
    r, c = np.concatenate(rows), np.concatenate(cols)
    adj = coo_matrix((np.ones(r.size, dtype=np.int8), (r, c)), shape=(N3, N3))
    ncomp, labels = connected_components(adj, directed=False)
    return int(ncomp), labels


def grain_statistics(grain_id, n, dx=1.0):
    """Number of grains (connected components, see grain_components) and their mean equivalent-sphere
    diameter (the mean over grains of (6 V / pi)^(1/3), same length unit as dx)."""
    ng, labels = grain_components(grain_id, n)
    vol = np.bincount(labels, minlength=ng).astype(np.float64) * dx ** 3
    return ng, float(np.mean((6.0 * vol / math.pi) ** (1.0 / 3.0)))
