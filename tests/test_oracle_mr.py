"""Pins of the oracle's Ma-Roters dislocation law (Sec. 2.2) against facts fixed by crystallography,
by mathematics and by the paper's equations read term by term.

- The |cos| / |sin| tables of Eqs. RhoForest / RhoParallel against values derived by hand for the
  FCC {111}<110> systems (t = n x d is a <112> direction);
- the projections of uniform densities against their closed forms;
- the flow rule (Eq. FlowRule) by its limits, its derivative and its potential, and the frozen
  hardening by its scaling laws and its Arrhenius factor;
- each term of Eq. SSDEvolution isolated by switching the others off;
- the GND stencil (Eq. GNDEvolution) on fields whose gradient is known exactly, with the one-sided
  differences at grain boundaries, against hand-derived slip geometry;
- the von Mises measures and Eq. L0evolution on textbook strain / stress states;
- the full-state update against the point model of a uniform crystal (a different solver), the
  softening of Eq. UpdateGND and the total density of Eq. TotDislocationDensity.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1509_04953_gb300 import synth

KB = 1.380649e-23
R2, R3, R6, R7 = math.sqrt(2.0), math.sqrt(3.0), math.sqrt(6.0), math.sqrt(7.0)


@pytest.fixture(scope="module")
def mat():
    return synth.ma_roters_material()


def _sorted_row(row):
    return np.sort(np.round(row, 12))


def test_projection_tables_are_the_fcc_angles():
    cNT, cND, sNT, sND = O.mr_tables()
    for a in range(12):
        cop = [b for b in range(12) if b // 3 == a // 3]          # the same {111} plane
        # n^a . t^b: 0 on the own plane; on each other plane one 4/(3 sqrt2) and two 2/(3 sqrt2)
        assert np.allclose(cNT[a, cop], 0.0, atol=1e-14)
        want = np.sort([0, 0, 0] + [4 / (3 * R2)] * 3 + [2 / (3 * R2)] * 6)
        assert np.allclose(_sorted_row(cNT[a]), want, atol=1e-12)
        # n^a . d^b: 0 on the own plane; on each other plane one 0 and two 2/sqrt6
        assert np.allclose(cND[a, cop], 0.0, atol=1e-14)
        assert np.allclose(_sorted_row(cND[a]), np.sort([0.0] * 6 + [2 / R6] * 6), atol=1e-12)
        # the sines of the same angles
        assert np.allclose(_sorted_row(sNT[a]), np.sort([1, 1, 1] + [1 / 3] * 3 + [R7 / 3] * 6), atol=1e-12)
        assert np.allclose(_sorted_row(sND[a]), np.sort([1.0] * 6 + [1 / R3] * 6), atol=1e-12)


def test_projection_closed_forms():
    rho = 3.7e11
    rF, rP = O.mr_project(np.full(12, rho))
    assert np.allclose(rF, 4 * R2 * rho, rtol=1e-14)
    assert np.allclose(rP, (4 + 2 * R7) * rho, rtol=1e-14)
    # signed GND components enter by magnitude; screw-like rho_GNDs projects with d, rho_GNDet with t
    g = -2.0e11
    rF, rP = O.mr_project(np.zeros(12), gs=np.full(12, g))
    assert np.allclose(rF, 2 * R6 * abs(g), rtol=1e-14)
    assert np.allclose(rP, (6 + 2 * R3) * abs(g), rtol=1e-14)
    rF, rP = O.mr_project(np.zeros(12), ge=np.full(12, g))
    assert np.allclose(rF, 4 * R2 * abs(g), rtol=1e-14)
    assert np.allclose(rP, (4 + 2 * R7) * abs(g), rtol=1e-14)
    # one density on one system: forest on the systems that see it, nothing on its own plane
    ssd = np.zeros(12)
    ssd[0] = 1.0e12
    rF, rP = O.mr_project(ssd)
    assert np.allclose(rF[:3], 0.0) and np.allclose(rP[:3], 1.0e12)


def test_flow_rule_limits_derivative_and_potential():
    tp, tcut, A = 11.0, 0.7, 2.5e-7
    for tau in (0.0, 5.0, 11.0, -11.0):
        g, dg, psi = O.mr_gdot(tau, tp, tcut, A)
        assert g == 0.0 and dg == 0.0 and psi == 0.0             # below the passing stress
    # sinh(asinh 1) = 1: at |tau| = tp + tcut asinh(1) the rate is exactly the prefactor
    g, _, _ = O.mr_gdot(tp + tcut * math.asinh(1.0), tp, tcut, A)
    assert g == pytest.approx(A, rel=1e-14)
    for tau in (12.3, 15.0, 18.0):
        g, dg, psi = O.mr_gdot(tau, tp, tcut, A)
        gm, _, _ = O.mr_gdot(-tau, tp, tcut, A)
        assert gm == -g                                           # odd in tau
        h = 1e-6
        gp, _, pp = O.mr_gdot(tau + h, tp, tcut, A)
        gq, _, pq = O.mr_gdot(tau - h, tp, tcut, A)
        assert dg == pytest.approx((gp - gq) / (2 * h), rel=1e-6)
        assert g == pytest.approx((pp - pq) / (2 * h), rel=1e-6)  # the potential's derivative is the rate
        assert psi > 0.0


def test_frozen_hardening_scaling_and_arrhenius(mat):
    rF = np.full(12, 1.0e12)
    rP = np.full(12, 2.0e12)
    tp, tcut, A = O.mr_frozen(mat, rF, rP)
    tp4, tcut4, A4 = O.mr_frozen(mat, 4 * rF, 4 * rP)
    assert np.allclose(tp4, 2 * tp) and np.allclose(tcut4, 2 * tcut) and np.allclose(A4, 2 * A)
    # tau_pass depends on rho_P only and tau_cut on rho_F only
    tpa, tcuta, Aa = O.mr_frozen(mat, 9 * rF, rP)
    assert np.allclose(tpa, tp) and np.allclose(tcuta, 3 * tcut) and np.allclose(Aa, A)
    # the prefactor is 2 k_B T nu_D sqrt(rho_P) exp(-Q_slip/k_B T) / (c1 c3 mu b^2): T exp(-Q/kT)
    hot, cold = synth.Material(T=800.0), synth.Material(T=600.0)
    A1 = O.mr_frozen(hot, rF, rP)[2][0]
    A2 = O.mr_frozen(cold, rF, rP)[2][0]
    assert A1 / A2 == pytest.approx(800.0 / 600.0 * math.exp(-mat.Q_slip / KB * (1 / 800.0 - 1 / 600.0)),
                                    rel=1e-12)
    assert np.allclose(O.mr_frozen(hot, rF, rP)[0], tp)         # athermal passing stress
    # the mobile density closure is proportional to T sqrt(rho_P rho_F)
    m1 = O.mr_rho_m(mat, 1.0e12, 2.0e12)
    assert O.mr_rho_m(mat, 4.0e12, 2.0e12) == pytest.approx(2 * m1, rel=1e-14)
    assert O.mr_rho_m(hot, 1.0e12, 2.0e12) / O.mr_rho_m(cold, 1.0e12, 2.0e12) == pytest.approx(800 / 600)


def _only(mat, **keep):
    """A copy of mat with the SSD constants c4..c7 switched off except those given."""
    kw = dict(c4=0.0, c5=0.0, c6=0.0, c7=0.0)
    kw.update(keep)
    m = synth.ma_roters_material()
    for k, v in kw.items():
        setattr(m, k, v)
    return m


def test_ssd_terms_one_by_one(mat):
    rng = np.random.default_rng(3)
    ssd = rng.uniform(1e11, 1e12, 12)
    rF = rng.uniform(1e12, 3e12, 12)
    rP = rng.uniform(1e12, 3e12, 12)
    tau = rng.uniform(-30, 30, 12)
    gd = rng.uniform(-1e-3, 1e-3, 12)
    gd[3] = 0.0
    # athermal annihilation: -c5 rho |gdot|, blind to the sign of slip
    r = O.mr_ssd_rate(_only(mat, c5=10.0), ssd, rF, rP, tau, gd, 50.0, 1e-3)
    assert np.allclose(r, -10.0 * ssd * np.abs(gd), rtol=1e-14)
    # lock formation: c4 sqrt(rho_F) |gdot|
    r1 = O.mr_ssd_rate(_only(mat, c4=8e7), ssd, rF, rP, tau, gd, 50.0, 1e-3)
    r4 = O.mr_ssd_rate(_only(mat, c4=8e7), ssd, 4 * rF, rP, tau, gd, 50.0, 1e-3)
    assert np.all(r1 >= 0) and r1[3] == 0.0 and np.allclose(r4, 2 * r1)
    assert np.allclose(r1, O.mr_ssd_rate(_only(mat, c4=8e7), ssd, rF, rP, tau, -gd, 50.0, 1e-3))
    # dipole formation: c6 d_dipole rho_M |gdot| with d_dipole inversely proportional to |tau|
    d1 = O.mr_ssd_rate(_only(mat, c6=3e10), ssd, rF, rP, tau, gd, 50.0, 1e-3)
    d2 = O.mr_ssd_rate(_only(mat, c6=3e10), ssd, rF, rP, 2 * tau, gd, 50.0, 1e-3)
    assert np.all(d1 >= 0) and d1[3] == 0.0 and np.allclose(d2, d1 / 2)
    rm = np.array([O.mr_rho_m(mat, rF[a], rP[a]) for a in range(12)])
    ddip = R3 * mat.mu * mat.b / (16 * math.pi * (1 - mat.poisson) * np.abs(tau))
    assert np.allclose(d1, 3e10 * ddip * rm * np.abs(gd), rtol=1e-12)
    # climb: -c7 exp(-Q_bulk/kT) |sigma_vm| / kT rho^2 gdot_vm^c8, on every system (gdot = 0 too)
    c1 = O.mr_ssd_rate(_only(mat, c7=7e-28), ssd, rF, rP, tau, gd, 50.0, 1e-3)
    assert np.all(c1 < 0) and c1[3] < 0
    assert np.allclose(O.mr_ssd_rate(_only(mat, c7=7e-28), 2 * ssd, rF, rP, tau, gd, 50.0, 1e-3), 4 * c1)
    assert np.allclose(O.mr_ssd_rate(_only(mat, c7=7e-28), ssd, rF, rP, tau, gd, 100.0, 1e-3), 2 * c1)
    assert np.allclose(O.mr_ssd_rate(_only(mat, c7=7e-28), ssd, rF, rP, tau, gd, 50.0, 2e-3),
                       2 ** 0.24 * c1, rtol=1e-12)
    kT = KB * mat.T
    want = -7e-28 * math.exp(-mat.Q_bulk / kT) * 50e6 / kT * ssd ** 2 * 1e-3 ** 0.24
    assert np.allclose(c1, want, rtol=1e-12)
    # all four together are the sum of the four
    tot = O.mr_ssd_rate(mat, ssd, rF, rP, tau, gd, 50.0, 1e-3)
    parts = (O.mr_ssd_rate(_only(mat, c4=mat.c4), ssd, rF, rP, tau, gd, 50.0, 1e-3) +
             O.mr_ssd_rate(_only(mat, c5=mat.c5), ssd, rF, rP, tau, gd, 50.0, 1e-3) + d1 + c1)
    assert np.allclose(tot, parts, rtol=1e-12)


def test_von_mises_measures():
    assert O.vm_stress([0, 0, -70.0, 0, 0, 0]) == pytest.approx(70.0, rel=1e-14)
    assert O.vm_stress([5.0, 5.0, 5.0, 0, 0, 0]) == pytest.approx(0.0, abs=1e-12)   # hydrostatic
    tau = 12.0
    assert O.vm_stress([0, 0, 0, 0, 0, R2 * tau]) == pytest.approx(R3 * tau, rel=1e-14)  # pure shear
    e = 2.0e-3
    assert O.vm_strain([-e / 2, -e / 2, e, 0, 0, 0]) == pytest.approx(e, rel=1e-14)   # isochoric uniaxial
    gam = 1e-3   # engineering shear: eps12 = gam / 2, Mandel sqrt2 eps12
    assert O.vm_strain([0, 0, 0, 0, 0, R2 * gam / 2]) == pytest.approx(gam / R3, rel=1e-14)
    assert O.mr_leff_next(21.4e-6, [-e / 2, -e / 2, e, 0, 0, 0], 200.0) == pytest.approx(21.4e-6 * (1 + e / 200))


def _slab_case(n, axis, width):
    """Grain 0 = the first `width` planes along `axis`, grain 1 the rest; a shear-rate field that is
    linear along `axis` inside each grain (a different slope per grain and per system)."""
    N3 = n ** 3
    idx = np.arange(N3)
    coord = np.stack([idx % n, (idx // n) % n, idx // (n * n)])[axis]
    g = np.where(coord < width, 0, 1).astype(np.int32)
    slopes = np.array([[1.0 + a, -2.0 + 0.5 * a] for a in range(12)]) * 1e-5   # per m of grid, per grain
    gd = np.zeros((12, N3))
    for a in range(12):
        gd[a] = 1e-4 * (a + 1) + slopes[a, g] * coord
    return g, gd, slopes, coord


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_gnd_stencil_exact_on_linear_fields(axis):
    n, b, leff = 8, 2.556e-10, 3.0
    quat = np.vstack([synth.axis_quaternion("001"), synth.axis_quaternion("z45")])
    g, gd, slopes, coord = _slab_case(n, axis, 3)
    rs, re = O.mr_gnd_rates(n, g, g, gd.reshape(-1), quat, leff, b)
    # hand-derived sample-frame vectors of system 0, plane (111), direction [0 1 -1]:
    # t = n x d = (-2, 1, 1)/sqrt6, d = (0, 1, -1)/sqrt2; grain 1 is turned 45 degrees about x3
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    t0 = np.array([-2.0, 1.0, 1.0]) / R6
    d0 = np.array([0.0, 1.0, -1.0]) / R2
    for gr, R in ((0, np.eye(3)), (1, Rz)):
        sel = g == gr
        grad = slopes[0, gr] / leff       # every voxel of the grain: central or one-sided, exact for a line
        assert np.allclose(rs[0, sel], -grad * (R @ t0)[axis] / b, rtol=1e-9, atol=1e-6)
        assert np.allclose(re[0, sel], grad * (R @ d0)[axis] / b, rtol=1e-9, atol=1e-6)
    # a grain one plane thick has no neighbour of its own along the axis: zero gradient
    g1, gd1, _, _ = _slab_case(n, axis, 1)
    rs1, re1 = O.mr_gnd_rates(n, g1, g1, gd1.reshape(-1), quat, leff, b)
    assert np.allclose(rs1[:, g1 == 0], 0.0) and np.allclose(re1[:, g1 == 0], 0.0)
    # a central difference across the boundary would see the jump between the grains' lines; the
    # rates are also inversely proportional to l_eff
    rs2, _ = O.mr_gnd_rates(n, g, g, gd.reshape(-1), quat, 2 * leff, b)
    assert np.allclose(rs2, rs / 2)


def test_same_grain_id_with_another_orientation_is_a_boundary():
    n, b, leff = 8, 2.556e-10, 1.0
    quat = np.vstack([synth.axis_quaternion("001"), synth.axis_quaternion("z45")])
    g, gd, slopes, coord = _slab_case(n, 0, 4)
    gcur = np.zeros_like(g)                         # one current grain id over both orientations
    rs, _ = O.mr_gnd_rates(n, gcur, g, gd.reshape(-1), quat, leff, b)
    rs_ref, _ = O.mr_gnd_rates(n, g, g, gd.reshape(-1), quat, leff, b)
    assert np.allclose(rs, rs_ref)


def test_newton_elastic_limit_and_converged_residual(mat):
    q = synth.axis_quaternion("z45")
    Cm, S, M = O.grain_tables(mat, q)
    rF, rP = O.mr_project(np.full(12, mat.rho0))
    tp, tcut, A = O.mr_frozen(mat, rF, rP)
    # below the passing stress the local problem is Hooke's law
    etr = np.array([1e-5, -2e-5, 0.5e-5, 1e-6, 0, 2e-6])
    rc, sig, gd, its = O.newton_mr(mat, S[0], M[0], etr, tp, tcut, A, tp.min(), 0.625, np.zeros(6))
    assert rc == 0 and np.all(gd == 0.0)
    assert np.allclose(sig, Cm[0] @ etr, rtol=1e-10)
    # far above it: the converged stress zeroes the residual and slips
    etr = np.array([2e-4, 2e-4, -8e-4, 1e-4, -5e-5, 3e-5])
    rc, sig, gd, its = O.newton_mr(mat, S[0], M[0], etr, tp, tcut, A, tp.min(), 0.625, np.zeros(6))
    assert rc == 0 and np.abs(gd).max() > 0
    r = O.residual_mr(mat, S[0], M[0], etr, tp, tcut, A, 0.625, sig)
    assert np.linalg.norm(r) < 1e-12 * np.linalg.norm(etr)
    taus = M[0] @ sig
    act = np.abs(taus) > tp
    assert np.all(np.abs(taus[act]) - tp[act] < 30 * tcut[act])     # resolved stresses near the threshold


def test_point_model_mr_elastic_start_and_flow_stress(mat):
    q = synth.axis_quaternion("001")
    _, S, M = O.grain_tables(mat, q)
    rc, hist, _ = O.point_model_mr(mat, S[0], M[0], -1e-5, 0.625, 1)
    # <001> Young's modulus of a cubic crystal (textbook): (C11 - C12)(C11 + 2 C12) / (C11 + C12)
    E001 = (mat.C11 - mat.C12) * (mat.C11 + 2 * mat.C12) / (mat.C11 + mat.C12)
    assert rc == 0 and hist[0] == pytest.approx(-E001 * 1e-5, rel=1e-9)
    rc, hist, st = O.point_model_mr(mat, S[0], M[0], -1e-3, 0.625, 20)
    # copper at 723 K, 1.6e-3 /s: tens of MPa, hardening (unit errors would be orders off)
    assert rc == 0 and -150.0 < hist[-1] < -20.0 and np.all(np.diff(hist) < 0)
    # <001> compression: the eight systems with Schmid factor 1/sqrt6 store dislocations, the four
    # with none lose a little by climb
    taus = M[0] @ np.array([0, 0, -1.0, 0, 0, 0])
    act = np.abs(taus) > 1e-12
    assert act.sum() == 8 and np.all(st["ssd"][act] > 3 * mat.rho0) and np.all(st["ssd"][~act] < mat.rho0)


def _poly(n, G, seed):
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, seed))
    return g0, synth.orientations(G, seed)


@pytest.mark.parametrize("scheme", [0, 1])
def test_uniform_crystal_matches_point_model_mr(mat, scheme):
    q = synth.axis_quaternion("z45")
    _, S, M = O.grain_tables(mat, q)
    _, hist, pm = O.point_model_mr(mat, S[0], M[0], -1e-3, 0.625, 4)
    n = 4
    st = O.State(n, 1, np.zeros(n ** 3, np.int32), q, mat, 5, law=1, tol=1e-11, newton_tol=1e-13, scheme=scheme,
                 al_scale=8.0, max_iter=4000)
    for t in range(4):
        rc, s = st.increment(-1e-3, 0.625)
        assert rc == 0
        assert s.sig_mean[2] == pytest.approx(hist[t], rel=1e-7)
    assert np.allclose(st.field("rho"), pm["ssd"][:, None], rtol=1e-7)
    assert np.allclose(st.field("gnd"), 0.0) and np.allclose(st.field("gnds"), 0.0)


def test_initial_total_density_closed_form(mat):
    n, G = 4, 2
    g0, quat = _poly(n, G, 2)
    st = O.State(n, G, g0, quat, mat, 3, law=1)
    rm = 2 * KB * mat.T / (mat.c1 * mat.c2 * mat.c3 * 1e6 * mat.mu * mat.b ** 3) * math.sqrt(
        4 * R2 * (4 + 2 * R7)) * mat.rho0
    assert np.allclose(st.field("k"), 12 * (mat.rho0 + rm), rtol=1e-13)
    assert st.leff == mat.dx


def _voxel_rates(st, mat, hard):
    """Shear rates of every voxel from the converged stress and the frozen hardening (numpy loops)."""
    M = O.grain_tables(mat, st._q.reshape(-1, 4))[2]
    sig = st.field("sig")
    g0 = st.ifield("g0")
    gd = np.zeros((12, st.N3))
    for v in range(st.N3):
        taus = M[g0[v]] @ sig[:, v]
        tp, tcut, A = hard[v]
        for a in range(12):
            gd[a, v] = O.mr_gdot(taus[a], tp[a], tcut[a], A[a])[0]
    return gd


def test_state_update_wires_the_gnd_and_ssd_laws(mat):
    n, G = 8, 4
    g0, quat = _poly(n, G, 9)
    st = O.State(n, G, g0, quat, mat, 7, law=1, tol=1e-9, newton_tol=1e-13, scheme=1, al_scale=8.0)
    assert st.increment(-1e-3, 0.625)[0] == 0
    rho0 = st.field("rho").copy()
    gs0, ge0, gnd0 = st.field("gnds").copy(), st.field("gndet").copy(), st.field("gnd").copy()
    leff0 = st.leff
    hard = []
    for v in range(st.N3):
        rF, rP = O.mr_project(rho0[:, v], gs0[:, v], ge0[:, v])
        hard.append(O.mr_frozen(mat, rF, rP))
    rc, s = st.increment(-1e-3, 0.625)
    assert rc == 0
    gd = _voxel_rates(st, mat, hard)
    rs, re = O.mr_gnd_rates(n, st.ifield("g"), g0, gd.reshape(-1), quat, leff0, mat.b)
    dt = 0.625
    assert np.allclose(st.field("gnds"), gs0 + dt * rs, rtol=1e-9, atol=1e3)
    assert np.allclose(st.field("gndet"), ge0 + dt * re, rtol=1e-9, atol=1e3)
    assert np.allclose(st.field("gnd"), gnd0 + dt * np.hypot(rs, re), rtol=1e-9, atol=1e3)
    assert np.abs(rs).max() > 1e9                                   # boundaries build GND
    assert st.leff == pytest.approx(O.mr_leff_next(leff0, st.field("E"), mat.xi), rel=1e-15)
    # k = sum of mobile, SSD and GND densities at the updated state
    for v in (0, 77, 300):
        rF, rP = O.mr_project(st.field("rho")[:, v], st.field("gnds")[:, v], st.field("gndet")[:, v])
        k = sum(O.mr_rho_m(mat, rF[a], rP[a]) for a in range(12)) + st.field("rho")[:, v].sum() + \
            st.field("gnd")[:, v].sum()
        assert st.field("k")[0, v] == pytest.approx(k, rel=1e-13)


def test_schemes_reach_the_same_mr_solution(mat):
    n, G = 8, 4
    g0, quat = _poly(n, G, 4)
    out = []
    for scheme in (0, 1):
        st = O.State(n, G, g0, quat, mat, 7, law=1, tol=1e-10, newton_tol=1e-13, scheme=scheme, al_scale=8.0,
                     max_iter=5000)
        for _ in range(2):
            assert st.increment(-1e-3, 0.625)[0] == 0
        out.append((st.field("sig").copy(), st.field("gnd").copy()))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-6 * np.abs(out[0][0]).max()
    assert np.allclose(out[0][1], out[1][1], rtol=1e-5, atol=1e-6 * out[0][1].max())


def test_nucleation_softens_gnd_and_keeps_ssd(mat):
    n, G = 8, 4
    g0, quat = _poly(n, G, 6)
    st = O.State(n, G, g0, quat, mat, 7, law=1, tol=1e-9, newton_tol=1e-13, scheme=1, al_scale=8.0)
    for _ in range(2):
        assert st.increment(-1e-3, 0.625)[0] == 0
    before = {f: st.field(f).copy() for f in ("rho", "gnds", "gndet", "gnd", "k")}
    st.field("kappa")[:] = 0.0                                     # every boundary voxel nucleates
    rc, nn = st.nucleate(0)
    assert rc == 0 and nn > 0
    new = st.ifield("g") >= G
    f = mat.s_soften
    assert np.array_equal(st.field("rho"), before["rho"])
    for name in ("gnds", "gndet", "gnd"):
        assert np.allclose(st.field(name)[:, new], f * before[name][:, new], rtol=1e-15)
        assert np.array_equal(st.field(name)[:, ~new], before[name][:, ~new])
    assert np.all(st.field("k")[0, new] < before["k"][0, new])
