"""Pins of the oracle's 2:1 phase-field grid (Sec. 2.4: the PF grid is refined 2:1 over the
FFT-EVP grid; smooth fields are interpolated linearly, orientations come from the nearest original
grid point, and the grain id after the PF steps is the argmax of the order parameters).

Readings pinned here: cell-centred periodic grids (PF cell I has its centre at I/2 + 1/4 in
mechanics-cell units), trilinear weights 3/4 (parent) and 1/4 (the neighbour on the side of the PF
centre), the grain id of a mechanics cell = argmax of the order parameters summed over its eight
children (ties to the smaller id), and PF lengths in PF grid spacings (dx / 2), so that the stored
energy per unit rho_tot halves with the spacing."""
import numpy as np
import pytest

import oracle as O
from paper_1509_04953_gb300 import synth


def refined(mat, n, G, seed=4, kmax=8):
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, seed))
    return O.State(n, G, g0, synth.orientations(G, seed), mat, seed=0, kmax=kmax, pf_refine=2), g0


def parent(n, w):
    m = 2 * n
    X, Y, Z = w % m, (w // m) % m, w // (m * m)
    return X // 2 + n * (Y // 2 + n * (Z // 2))


def set_k(st, kfield):
    """Set rho so that rho_tot equals kfield (rho split evenly; 12 equal dyadic parts sum exactly)."""
    st.field("rho")[:] = np.asarray(kfield, dtype=np.float64)[None, :] / 12.0
    O.lib().orc_refresh_derived(st.h)


def test_initial_pf_points_take_the_parent_grain(mat):
    n, G = 8, 5
    st, g0 = refined(mat, n, G)
    w = np.arange((2 * n) ** 3)
    par = parent(n, w)
    ids, eta = st.ifield("ids"), st.field("eta")
    assert np.array_equal(ids[0], g0[par])
    assert np.all(eta[0] == 1.0) and np.all(ids[1:] == -1)
    assert np.array_equal(st.ifield("gpf"), g0[par])


def test_interpolation_constant_mean_and_linear_fields(mat):
    n = 8
    st, _ = refined(mat, n, 3)
    N3 = n ** 3
    set_k(st, np.full(N3, 12.0))
    assert np.all(st.field("kpf") == 12.0)                     # a constant is reproduced exactly
    rng = np.random.default_rng(3)
    kk = rng.uniform(1.0, 2.0, N3) * 12.0
    set_k(st, kk)
    # every mechanics value is spread with weights summing to 2 per axis: the mean is kept
    assert abs(st.field("kpf").sum() / (8.0 * st.field("k").sum()) - 1.0) < 1e-13
    x = np.arange(N3) % n
    set_k(st, 12.0 + 6.0 * x)                                  # linear along x (dyadic values)
    m = 2 * n
    X = np.arange(m ** 3) % m
    inner = (X >= 1) & (X <= m - 2)                            # stencils that do not wrap
    want = 12.0 + 6.0 * (X / 2.0 - 0.25)                       # the field at the PF centres
    assert np.array_equal(st.field("kpf")[inner], want[inner])
    # the periodic wrap: PF cell 0 lies between mechanics cells n-1 (weight 1/4) and 0 (3/4)
    k = st.field("k")[0]
    assert st.field("kpf")[0] == 0.25 * k[n - 1] + 0.75 * k[0]


def test_restriction_recovers_grains_and_takes_the_larger_sum(mat):
    n, G = 4, 3
    st, g0 = refined(mat, n, G, seed=2)
    st.pf_step_dense(0)                                        # rewrite + argmax + restriction
    assert np.array_equal(st.ifield("g"), g0)
    m = 2 * n
    ids, eta = st.ifield("ids"), st.field("eta")
    kids = [(2 * 0 + (c & 1)) + m * ((2 * 0 + ((c >> 1) & 1)) + m * (2 * 0 + (c >> 2))) for c in range(8)]
    # five children of cell 0 hold grain 2 (eta 0.6), three hold grain 1 (eta 0.9): 3.0 > 2.7
    for c, w in enumerate(kids):
        ids[:, w] = -1
        eta[:, w] = 0.0
        ids[0, w] = 2 if c < 5 else 1
        eta[0, w] = 0.6 if c < 5 else 0.9
    st.pf_step_dense(0)
    assert st.ifield("g")[0] == 2
    # equal sums: the smaller id wins
    for c, w in enumerate(kids):
        ids[0, w] = 2 if c < 4 else 1
        eta[0, w] = 0.5
    st.pf_step_dense(0)
    assert st.ifield("g")[0] == 1


def test_refined_sparse_active_set_equals_dense_bitwise(mat):
    import dataclasses
    m2 = dataclasses.replace(mat, eta_drop=-1e300)
    n, G = 4, 3
    a, g0 = refined(m2, n, G, seed=4, kmax=16)
    b, _ = refined(m2, n, G, seed=4, kmax=16)
    Esc = mat.zeta * mat.mu * 1e6 * mat.b ** 2 * mat.dx / mat.omega_gb
    for s in (a, b):
        set_k(s, np.linspace(0.2, 1.2, n ** 3) / Esc)
        ids = s.ifield("ids")
        ids[0, 37] = G
        ids[0, 300] = G + 1
        s.next_id = G + 2
    a.pf_step(4)
    b.pf_step_dense(4)
    assert np.array_equal(a.ifield("gpf"), b.ifield("gpf"))
    assert np.array_equal(a.ifield("g"), b.ifield("g"))
    ia, ib = a.ifield("ids"), b.ifield("ids")
    ea, eb = a.field("eta"), b.field("eta")
    for v in range((2 * n) ** 3):
        da = {int(i): ea[j, v] for j, i in enumerate(ia[:, v]) if i >= 0 and ea[j, v] != 0.0}
        db = {int(i): eb[j, v] for j, i in enumerate(ib[:, v]) if i >= 0}
        assert da == db


def test_nucleus_fills_its_eight_pf_children(mat):
    n, G = 8, 4
    st, g0 = refined(mat, n, G)
    N3 = n ** 3
    g = g0.reshape(n, n, n)
    bnd = np.zeros_like(g, dtype=bool)
    for ax in range(3):
        for sh in (1, -1):
            bnd |= g != np.roll(g, sh, axis=ax)
    v = int(np.flatnonzero(bnd.reshape(-1))[0])
    kappa = st.field("kappa")
    kappa[:] = 1e300
    kappa[0, v] = 0.5 * st.field("k")[0, v]
    rc, nn = st.nucleate(0)
    assert rc == 0 and nn == 1
    assert st.ifield("g")[v] == G
    m = 2 * n
    x, y, z = v % n, (v // n) % n, v // (n * n)
    ids, eta = st.ifield("ids"), st.field("eta")
    for c in range(8):
        w = (2 * x + (c & 1)) + m * ((2 * y + ((c >> 1) & 1)) + m * (2 * z + (c >> 2)))
        assert ids[0, w] == G and eta[0, w] == 1.0 and np.all(ids[1:, w] == -1)
        assert st.ifield("gpf")[w] == G
    assert np.count_nonzero(st.ifield("gpf") == G) == 8
    # densities of the nucleus cell softened, and the PF driving force re-interpolated from them
    assert st.field("k")[0, v] < 12 * mat.rho0


def test_refined_boundary_velocity_uses_the_pf_spacing(mat):
    """A flat rex/def boundary on the refined grid moves M E'_pf PF spacings per unit PF time with
    E'_pf = zeta mu b^2 rho_tot (dx / 2) / omega_gb, half the mechanics-grid value for the same density."""
    n = 16
    x = np.arange(n ** 3) % n
    g0 = (x >= n // 3 + 1).astype(np.int32)
    st = O.State(n, 2, g0, synth.orientations(2, 0), mat, seed=0, kmax=8, pf_refine=2)
    ids = st.ifield("ids")
    ids[0][ids[0] == 0] = 2
    st.ifield("gpf")[:] = ids[0]
    st.ifield("g")[:] = np.where(g0 == 0, 2, g0)
    st.next_id = 3
    set_k(st, np.zeros(n ** 3))
    st.pf_step(60)                                             # relax the sharp start
    Ep = 0.3
    Esc_pf = mat.zeta * mat.mu * 1e6 * mat.b ** 2 * (mat.dx / 2) / mat.omega_gb
    set_k(st, np.full(n ** 3, Ep / Esc_pf))
    dt_step = mat.L_dt * 3.0 * mat.l_gb / 4.0
    m = 2 * n

    def rex_width():
        ids, eta = st.ifield("ids"), st.field("eta")
        return sum(eta[:, X][ids[:, X] == 2].sum() for X in range(m))
    st.pf_step(20)
    w0 = rex_width()
    steps = 200
    st.pf_step(steps)
    w1 = rex_width()
    v = (w1 - w0) / 2.0 / (steps * dt_step)
    assert abs(v / Ep - 1.0) < 0.08
