"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks one part of the oracle against something other than itself: a definition
written out independently (brute-force DFT, brute-force Voronoi), a closed form (elastic
modulus of a <001> crystal, rotated cubic constants, the Kocks-Mecking ODE solution, the
non-hardening steady state, the layered laminate, the tanh interface profile), an invariant
(idempotent Green projection, divergence-free polarisation, monotone free energy) or a
statistical law (Weibull CDF of the nucleation strength, Eqs. NumCrt / NuclStrengthProb).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1509_04953_gb300 import synth

SQ2 = math.sqrt(2.0)
MI = [0, 1, 2, 1, 0, 0]
MJ = [0, 1, 2, 2, 2, 1]


def m2t(v):
    """Mandel 6-vector -> symmetric 3x3 tensor (written here, independent of the oracle)."""
    T = np.zeros((3, 3), dtype=np.result_type(v, float))
    for I in range(6):
        w = 1.0 if I < 3 else SQ2
        T[MI[I], MJ[I]] = v[I] / w
        T[MJ[I], MI[I]] = v[I] / w
    return T


def t2m(T):
    return np.array([T[0, 0], T[1, 1], T[2, 2], SQ2 * T[1, 2], SQ2 * T[0, 2], SQ2 * T[0, 1]])


def C0_mandel(lam, mu):
    C = 2.0 * mu * np.eye(6)
    C[:3, :3] += lam
    return C


# ------------------------------------------------------------------------------------------
# hash + Weibull (Sec. 2.3, Eqs. NumCrt / NuclStrengthProb; SplitMix64)
# ------------------------------------------------------------------------------------------
def test_splitmix64_published_vector():
    # first three outputs of SplitMix64 started from state 0 (golden-gamma increments)
    g = 0x9E3779B97F4A7C15
    want = [int(x, 16) for x in open(__file__.replace("test_oracle_pins.py", "golden/splitmix64.txt"))
            .read().split("#")[0].split()]
    got = [O.lib().orc_mix64((k * g) & (2 ** 64 - 1)) for k in (1, 2, 3)]
    assert got == want


def test_weibull_sampler_matches_cdf(mat):
    scipy_stats = pytest.importorskip("scipy.stats")
    n = 200000
    L = O.lib()
    kap = np.array([L.orc_weibull(L.orc_u01(12345, i, 0), mat.kc, mat.q) for i in range(n)])
    cdf = lambda k: 1.0 - np.exp(-(np.asarray(k) / mat.kc) ** mat.q)  # Eq. NumCrt
    res = scipy_stats.kstest(kap, cdf)
    assert res.pvalue > 1e-3
    assert abs(kap.mean() / (mat.kc * math.gamma(1.0 + 1.0 / mat.q)) - 1.0) < 5e-3
    u = np.array([L.orc_u01(7, i, 3) for i in range(20000)])
    assert 0.0 < u.min() and u.max() < 1.0
    assert scipy_stats.kstest(u, "uniform").pvalue > 1e-3


def test_nucleation_fraction_and_bookkeeping(mat):
    """Uniform k on all-boundary voxels: the nucleated fraction is 1-exp(-(k/kc)^q)."""
    n, G = 32, 2
    x = np.arange(n ** 3) % n
    g0 = (x % 2).astype(np.int32)                      # every voxel has a differing x-neighbour
    q = synth.orientations(G, 3)
    st = O.State(n, G, g0, q, mat, seed=99)
    P = 0.3
    kstar = mat.kc * (-math.log(1.0 - P)) ** (1.0 / mat.q)
    k = st.field("k")
    k[:] = kstar
    rho_before = st.field("rho").copy()
    rc, nn = st.nucleate(0)
    frac = nn / n ** 3
    assert abs(frac - P) < 5.0 * math.sqrt(P * (1 - P) / n ** 3)
    g = st.ifield("g")
    new = np.nonzero(g >= G)[0]
    assert len(new) == nn
    assert np.array_equal(g[new], G + np.arange(nn))   # fresh ids in ascending voxel order
    rho = st.field("rho")
    assert np.allclose(rho[:, new], mat.s_soften * rho_before[:, new], rtol=1e-15)
    kap = st.field("kappa")
    L = O.lib()
    v = int(new[0])
    assert kap[0, v] == L.orc_weibull(L.orc_u01(99, v, 1), mat.s_nucl * mat.kc, mat.q)
    assert st.ifield("draws")[v] == 1
    assert st.next_id == G + nn


# ------------------------------------------------------------------------------------------
# microstructure
# ------------------------------------------------------------------------------------------
def _voronoi_brute(n, seeds):
    L = n << 16
    out = np.zeros((n, n, n), dtype=np.int64)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                c = np.array([(x << 16) + 32768, (y << 16) + 32768, (z << 16) + 32768], dtype=np.int64)
                d = np.abs(seeds - c) % L
                d = np.minimum(d, L - d)
                d2 = (d * d).sum(axis=1)
                out[z, y, x] = int(np.argmin(d2))     # argmin takes the first (smallest) index on a tie
    return out


def test_voronoi_brute_force():
    """Periodic Voronoi ids against brute force: random seeds, and seeds on voxel centres, where whole planes of
    voxels lie at equal distance from two or three seeds and reading C21 gives them the smaller seed index."""
    n, G = 8, 11
    seeds = synth.voronoi_seeds(n, G, 5)
    assert np.array_equal(O.voronoi(n, seeds).reshape(n, n, n), _voronoi_brute(n, seeds))
    c = lambda i: (i << 16) + 32768
    tied = np.array([[c(2), c(0), c(0)], [c(0), c(0), c(0)], [c(0), c(2), c(0)]], dtype=np.int64)
    want = _voronoi_brute(4, tied)
    assert want[0, 0, 1] == 0 and want[0, 0, 3] == 0 and want[0, 1, 1] == 0   # ties to seeds 0 and 1, and 0, 1, 2
    assert np.array_equal(O.voronoi(4, tied).reshape(4, 4, 4), want)


def test_rotation_and_slip_geometry():
    h = 0.3
    R = O.quat_to_R([math.cos(h / 2), 0, 0, math.sin(h / 2)])
    assert np.allclose(R, [[math.cos(h), -math.sin(h), 0], [math.sin(h), math.cos(h), 0], [0, 0, 1]], atol=1e-15)
    q = synth.orientations(5, 1)
    for qq in q:
        R = O.quat_to_R(qq)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14) and abs(np.linalg.det(R) - 1) < 1e-14
    d, nr = O.slip_systems()
    assert np.allclose((d * nr).sum(1), 0) and np.allclose(np.linalg.norm(d, axis=1), 1)
    assert len({tuple(np.round(np.sign(v[0]) * v * math.sqrt(3), 6)) for v in nr}) == 4


def test_grain_tables_closed_forms(mat):
    C11, C12, C44 = mat.C11, mat.C12, mat.C44
    C, S, M = O.grain_tables(mat, [[1, 0, 0, 0]])
    want = np.zeros((6, 6))
    want[:3, :3] = C12
    np.fill_diagonal(want[:3, :3], C11)
    want[3, 3] = want[4, 4] = want[5, 5] = 2 * C44
    assert np.allclose(C[0], want, rtol=1e-14, atol=1e-9)
    den = (C11 - C12) * (C11 + 2 * C12)
    assert abs(S[0, 0, 0] - (C11 + C12) / den) < 1e-18 and abs(S[0, 0, 1] + C12 / den) < 1e-18
    # 45 degrees about x3: C'11 = (C11+C12)/2 + C44, C'12 = (C11+C12)/2 - C44, C'66 = (C11-C12)/2
    C45, _, _ = O.grain_tables(mat, synth.axis_quaternion("z45"))
    c = C45[0]
    assert abs(c[0, 0] - ((C11 + C12) / 2 + C44)) < 1e-8
    assert abs(c[0, 1] - ((C11 + C12) / 2 - C44)) < 1e-8
    assert abs(c[5, 5] / 2 - (C11 - C12) / 2) < 1e-8
    assert abs(c[2, 2] - C11) < 1e-8
    # Schmid tensors: traceless, |m|^2 = 1/2, and on <001> uniaxial stress 8 systems carry 1/sqrt6
    m = M[0]
    assert np.allclose(m[:, :3].sum(1), 0, atol=1e-15)
    assert np.allclose((m * m).sum(1), 0.5)
    tau = m @ np.array([0, 0, 1.0, 0, 0, 0])
    assert sorted(np.round(np.abs(tau) * math.sqrt(6), 12)) == [0.0] * 4 + [1.0] * 8


# ------------------------------------------------------------------------------------------
# P1 FFT
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 8])
def test_fft_matches_brute_dft(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    for sign in (-1, 1):
        f = O.fft3d(a, sign)
        b = O.dft3d_brute(a, sign)
        assert np.abs(f - b).max() < 1e-12 * np.abs(b).max()


def test_fft1d_against_numpy():
    rng = np.random.default_rng(0)
    for n in (2, 16, 256):
        a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        assert np.allclose(O.fft1d(a, -1), np.fft.fft(a), rtol=1e-13, atol=1e-12)


# ------------------------------------------------------------------------------------------
# P2 Green operator
# ------------------------------------------------------------------------------------------
def test_gamma0_projection_properties(mat):
    lam, mu = mat.lam, mat.mu
    C0 = C0_mandel(lam, mu)
    rng = np.random.default_rng(1)
    for _ in range(20):
        xi = rng.standard_normal(3)
        Gm = O.gamma0(xi, lam, mu)
        assert np.allclose(Gm, Gm.T, rtol=1e-13, atol=1e-20)
        assert np.allclose(Gm @ C0 @ Gm, Gm, rtol=1e-12, atol=1e-18)            # idempotent
        u = rng.standard_normal(3)
        eps_c = t2m(0.5 * (np.outer(xi, u) + np.outer(u, xi)))                 # compatible strain
        assert np.allclose(Gm @ C0 @ eps_c, eps_c, rtol=1e-12, atol=1e-15)
        tau = rng.standard_normal(6)
        pol = C0 @ (Gm @ tau) - tau                                            # equilibrated
        assert np.abs(m2t(pol) @ xi).max() < 1e-12 * np.abs(tau).max() * np.linalg.norm(xi)
    assert np.allclose(O.gamma0([2.0, -1.0, 0.5], lam, mu), O.gamma0([-4.0, 2.0, -1.0], lam, mu))


# ------------------------------------------------------------------------------------------
# P4 point model closed forms, P6 Newton, P7 KM ODE
# ------------------------------------------------------------------------------------------
def test_point_model_elastic_modulus(mat):
    import dataclasses
    m2 = dataclasses.replace(mat, tau0=1e9)
    _, S, M = O.grain_tables(m2, [[1, 0, 0, 0]])
    rc, hist, st = O.point_model(m2, S[0], M[0], -1e-3, 1.0, 1)
    C11, C12 = mat.C11, mat.C12
    E001 = (C11 - C12) * (C11 + 2 * C12) / (C11 + C12)
    assert rc == 0
    assert abs(hist[0] / -1e-3 / E001 - 1) < 1e-10
    assert abs(st["E"][0] / -1e-3 + C12 / (C11 + C12)) < 1e-10


def test_point_model_nonhardening_steady_state(mat):
    import dataclasses
    m2 = dataclasses.replace(mat, k1=0.0, k2=0.0)
    _, S, M = O.grain_tables(m2, [[1, 0, 0, 0]])
    rc, hist, _ = O.point_model(m2, S[0], M[0], -1e-3, 1.0, 40)
    tauc = mat.tau0 + mat.alpha * mat.mu * mat.b * math.sqrt(12 * mat.rho0)
    rate = 1e-3
    want = math.sqrt(6) * tauc * (math.sqrt(6) * rate / (8 * mat.gdot0)) ** (1 / mat.n)
    assert rc == 0
    assert abs(-hist[-1] / want - 1) < 1e-9


def test_newton_tangent_and_residual(mat):
    q = synth.orientations(3, 11)
    _, S, M = O.grain_tables(mat, q)
    rng = np.random.default_rng(2)
    tauc, dt = 30.0, 1.0
    for g in range(3):
        eps_tr = rng.standard_normal(6) * 2e-3
        sig = rng.standard_normal(6) * 20.0
        r, K = O.residual(mat, S[g], M[g], eps_tr, tauc, dt, sig)
        Kfd = np.zeros((6, 6))
        for j in range(6):
            h = 1e-5 * max(1.0, abs(sig[j]))
            sp, sm = sig.copy(), sig.copy()
            sp[j] += h
            sm[j] -= h
            Kfd[:, j] = (O.residual(mat, S[g], M[g], eps_tr, tauc, dt, sp)[0] -
                         O.residual(mat, S[g], M[g], eps_tr, tauc, dt, sm)[0]) / (2 * h)
        assert np.allclose(K, Kfd, rtol=1e-6, atol=1e-12 * np.abs(K).max())
        assert np.allclose(K, K.T, rtol=1e-12)
        assert np.all(np.linalg.eigvalsh(K) > 0)
        rc, s, gd, its = O.newton(mat, S[g], M[g], eps_tr, tauc, dt, np.zeros(6))
        assert rc == 0
        r, _ = O.residual(mat, S[g], M[g], eps_tr, tauc, dt, s)
        assert np.abs(r).max() < 1e-12 * np.abs(eps_tr).max() + 1e-16
        # stress-strain consistency: sigma = C:(eps_tr - dt * sum m gdot) (Eq. HookeLaw)
        Cg = np.linalg.inv(S[g])
        assert np.allclose(s, Cg @ (eps_tr - dt * (M[g].T @ gd)), rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("sense", [1.0, -1.0])
def test_km_single_system_closed_form(mat, sense):
    """The densities grow with the accumulated |shear|: the same closed form for either sense of slip."""
    gd = np.zeros(12)
    gd[0] = sense
    errs = []
    for steps in (2000, 4000):
        gam = 0.2
        dt = gam / steps
        rho = np.zeros(12)
        rho[0] = mat.rho0
        for _ in range(steps):
            rho = O.km_update(mat, rho, gd, dt)
        r = mat.k1 / mat.k2
        want = (r - (r - math.sqrt(mat.rho0)) * math.exp(-mat.k2 * gam / 2)) ** 2
        errs.append(abs(rho[0] / want - 1))
    assert errs[0] < 1e-3
    assert 1.6 < errs[0] / errs[1] < 2.4          # first-order convergence of the explicit step


# ------------------------------------------------------------------------------------------
# P3 homogeneous crystal = point model; P5 layered laminate
# ------------------------------------------------------------------------------------------
def test_homogeneous_crystal_matches_point_model(mat):
    n = 4
    q = synth.orientations(1, 21)
    g0 = np.zeros(n ** 3, dtype=np.int32)
    st = O.State(n, 1, g0, q, mat, seed=1, tol=1e-12, max_iter=20000)
    _, S, M = O.grain_tables(mat, q)
    rc, hist, pm = O.point_model(mat, S[0], M[0], -1e-3, 1.0, 6)
    for inc in range(6):
        rc, s = st.increment(-1e-3, 1.0)
        assert rc == 0
        assert abs(s.sig_mean[2] / hist[inc] - 1) < 1e-9
        assert max(abs(s.sig_mean[i]) for i in (0, 1, 3, 4, 5)) < 1e-9 * abs(hist[inc])
        sig = st.field("sig")
        assert np.abs(sig - sig.mean(axis=1, keepdims=True)).max() < 1e-10 * abs(hist[inc])
    assert np.allclose(np.array(s.E), pm["E"], rtol=1e-8, atol=1e-12)
    assert np.allclose(st.field("rho")[:, 0], pm["rho"], rtol=1e-9)


@pytest.mark.parametrize("n,G", [(16, 8), (32, 27)])
def test_converged_increment_checks_hold_for_the_oracle(mat, n, G):
    """The any-size checks that the GPU's full-size increment is held to (tests/increment_checks.py) hold for the
    oracle's own converged first increment to round-off: equilibrium within the tolerance, zero stress-controlled
    means, and at sampled voxels the local update, plastic strain, densities and k."""
    from increment_checks import check_first_increment
    seed = synth.BASE_SEED + 2
    quat = synth.orientations(G, seed)
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, seed))
    st = O.State(n, G, g0, quat, mat, seed=seed, tol=1e-6, max_iter=5000)
    rc, s = st.increment(-1e-3, 1.0)
    assert rc == 0
    fields = {f: st.field(f) for f in ("sig", "eps", "epsp", "rho")}
    fields["k"] = st.field("k")[0]
    sample = np.random.default_rng(3).choice(n ** 3, 200, replace=False)
    err = check_first_increment(mat, quat, g0, n, 1.0, 1e-6, fields, s.sig_mean, sample, 1e-9, 1e-9, eq_factor=1.0)
    assert err > 1e-8      # converged to the tolerance, not far below it
    # a wrong time step in the state update is caught
    with pytest.raises(AssertionError):
        check_first_increment(mat, quat, g0, n, 2.0, 1e-6, fields, s.sig_mean, sample, 1e-9, 1e-9)


def test_any_increment_checks_hold_for_the_oracle_in_the_drx_regime(mat):
    """The any-increment checks (tests/increment_checks.py check_increment) that the GPU's full-size run in the DRX
    regime is held to hold for the oracle's own run to round-off: densities raised so that nucleation and sweep
    softening act, two coupled increments, then the third increment checked from the state before it."""
    from increment_checks import check_increment
    n, G, seed = 16, 8, synth.BASE_SEED
    quat = synth.orientations(G, seed)
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, seed))
    st = O.State(n, G, g0, quat, mat, seed=seed, tol=1e-6, max_iter=5000)
    st.field("rho")[:] = np.repeat(np.random.default_rng(1).uniform(2e13, 6e13, size=(1, n ** 3)), 12, axis=0)
    st.refresh_derived()
    nuclei = 0
    for inc in range(2):
        assert st.increment(-1e-3, 1.0)[0] == 0
        nuclei += st.nucleate(inc)[1]
        st.pf_step(5)
    assert nuclei > 0
    before = {f: st.field(f).copy() for f in ("epsp", "rho")}
    rc, s = st.increment(-1e-3, 1.0)
    assert rc == 0
    after = {f: st.field(f) for f in ("sig", "eps", "epsp", "rho")}
    after["k"] = st.field("k")[0]
    sample = np.random.default_rng(4).choice(n ** 3, 200, replace=False)
    check_increment(mat, quat, g0, n, 1.0, 1e-6, before, after, s.sig_mean, sample, 1e-9, 1e-9, eq_factor=1.0)
    with pytest.raises(AssertionError):      # the densities before the increment, not after, freeze tau_c
        check_increment(mat, quat, g0, n, 1.0, 1e-6, {"epsp": before["epsp"], "rho": after["rho"]}, after,
                        s.sig_mean, sample, 1e-9, 1e-9)


@pytest.mark.parametrize("scheme,ref_scale", [(0, 1.0), (1, 1.0), (0, 1.3)],
                         ids=["basic", "augmented_lagrangian", "basic_softer_reference"])
def test_elastic_laminate_closed_form(mat, scheme, ref_scale):
    """P5 under every fixed-point variant: the basic scheme, the augmented Lagrangian (Sec. 2.1) and a softer
    isotropic reference medium all reach the laminate's closed-form strain and stress."""
    import dataclasses
    m2 = dataclasses.replace(mat, gdot0=0.0)
    n = 8
    q = synth.orientations(2, 31)
    z = np.arange(n ** 3) // (n * n)
    g0 = (z >= n // 2).astype(np.int32)
    st = O.State(n, 2, g0, q, m2, seed=1, tol=1e-13, max_iter=5000, scheme=scheme, al_scale=6.0,
                 ref_scale=ref_scale)
    E33 = -1e-3
    rc, s = st.increment(E33, 1.0)
    assert rc == 0
    C, _, _ = O.grain_tables(m2, q)
    # unknowns: E11, E22, E12 (Mandel slots 0,1,5) shared; per phase e33, e23, e13 (slots 2,3,4)
    A = np.zeros((9, 9))
    b = np.zeros(9)

    def eps_map(p):
        P = np.zeros((6, 9))
        P[0, 0] = P[1, 1] = P[5, 2] = 1
        P[2, 3 + 3 * p] = P[3, 4 + 3 * p] = P[4, 5 + 3 * p] = 1
        return P
    S1, S2 = C[0] @ eps_map(0), C[1] @ eps_map(1)
    row = 0
    for k in (2, 3, 4):           # traction continuity
        A[row] = S1[k] - S2[k]
        row += 1
    for k in (0, 1, 5):           # zero mean in-plane stress
        A[row] = 0.5 * (S1[k] + S2[k])
        row += 1
    for k in (3, 4):              # zero (uniform) shear tractions
        A[row] = S1[k]
        row += 1
    A[row, 3] = A[row, 6] = 0.5   # mean e33 prescribed
    b[row] = E33
    x = np.linalg.solve(A, b)
    eps = st.field("eps")
    for p in (0, 1):
        want = eps_map(p) @ x
        sel = g0 == p
        assert np.abs(eps[:, sel] - want[:, None]).max() < 1e-10 * abs(E33)
        sw = C[p] @ want
        assert np.abs(st.field("sig")[:, sel] - sw[:, None]).max() < 1e-9 * np.abs(sw).max()


# ------------------------------------------------------------------------------------------
# P9-P12 phase field
# ------------------------------------------------------------------------------------------
def slab_state(mat, n, width, rex=False, kmax=8):
    x = np.arange(n ** 3) % n
    g0 = (x >= width).astype(np.int32)
    st = O.State(n, 2, g0, synth.orientations(2, 0), mat, seed=0, kmax=kmax)
    st.field("k")[:] = 0.0
    if rex:   # the slab x < width becomes a recrystallised grain (id >= G)
        ids = st.ifield("ids")
        ids[0][ids[0] == 0] = 2
        st.ifield("g")[:] = ids[0]
        st.next_id = 3
    return st


def test_pf_flat_interface_tanh_profile_and_energy(mat):
    n = 16
    st = slab_state(mat, n, n // 2)
    for _ in range(6):
        st.pf_step(100)
    ids, eta = st.ifield("ids"), st.field("eta")
    prof = np.array([eta[:, x][ids[:, x] == 0].sum() for x in range(n)])   # line y=z=0
    x = np.arange(n) + 0.0
    l = mat.l_gb
    want = 0.5 * (1 - np.tanh(2 * (x - (n / 2 - 0.5)) / l)) + 0.5 * (1 + np.tanh(2 * (x - (n - 0.5)) / l)) \
        + 0.5 * (1 + np.tanh(2 * (x + 0.5) / l)) - 1.0
    assert np.abs(prof - want).max() < 0.02
    # energy per unit area of a flat boundary is omega_gb = 1 (nondimensional)
    F = st.pf_energy()
    assert abs(F / (2 * n * n) - 1.0) < 0.03


@pytest.mark.parametrize("lfac,tol", [(1.0, 0.08), (2.0, 0.02)])
def test_pf_boundary_velocity_is_mobility_times_driving_force(mat, lfac, tol):
    """Flat def/rex boundaries move at v = M * E' (M = 1 nondimensional). At the paper's
    interface width l_gb = sqrt(9.6) dx (Sec. 2.4) the grid costs about 6 %; at twice that width
    the discrete velocity converges to M * E' (the sharp-interface value)."""
    import dataclasses
    m2 = dataclasses.replace(mat, l_gb=mat.l_gb * lfac)
    n = 32 if lfac == 1.0 else 64
    st = slab_state(m2, n, n // 3 + 1, rex=True)
    st.pf_step(int(60 * lfac * lfac))               # relax the sharp start without driving force
    Ep = 0.3 / lfac
    Esc = m2.zeta * m2.mu * 1e6 * m2.b ** 2 * m2.dx / m2.omega_gb
    st.field("k")[:] = Ep / Esc
    dt_step = m2.L_dt * 3.0 * m2.l_gb / 4.0         # L dt with L = 4M/(3 l), M = 1

    def rex_width():
        ids, eta = st.ifield("ids"), st.field("eta")
        return sum(eta[:, x][ids[:, x] == 2].sum() for x in range(n))
    st.pf_step(20)
    w0 = rex_width()
    steps = int(200 * lfac)
    st.pf_step(steps)
    w1 = rex_width()
    v = (w1 - w0) / 2.0 / (steps * dt_step)         # two boundaries move apart
    assert abs(v / Ep - 1.0) < tol


def test_pf_sweep_softening_and_recrystallised_fraction(mat):
    """Reading C14 (Eq. UpdateGND applied to swept material) and the statistics of Sec. 2.4 on a moving flat
    rex/def slab: X_rex and n_grains of the start are the construction's (width/n, 2 grains); during one call the
    recrystallised slab grows; exactly the voxels whose grain turned from deformed to recrystallised have their
    densities scaled by s_soften, once, with k their sum; every other voxel keeps its densities bitwise; X_rex
    grows by the swept count over N^3; a second call does not soften those voxels again."""
    n, width = 32, 11
    st = slab_state(mat, n, width, rex=True)
    N3 = n ** 3
    rc, ps = st.pf_step(0)
    assert ps.n_grains == 2 and ps.X_rex == width / n
    st.pf_step(60)                                   # relax the sharp start (no stored energy yet)
    Esc = mat.zeta * mat.mu * 1e6 * mat.b ** 2 * mat.dx / mat.omega_gb
    v = np.arange(N3)
    pattern = (1.0 + np.arange(12)[:, None] / 12.0) * (1.0 + (v % 5)[None, :] / 10.0)
    rho = st.field("rho")
    rho[:] = pattern * (0.3 / Esc) / pattern.sum(axis=0)[None, :].mean()
    st.field("k")[0][:] = rho.sum(axis=0)
    G = 2
    g0 = st.ifield("g").copy()
    rho0 = rho.copy()
    _, ps0 = st.pf_step(0)
    rc, ps1 = st.pf_step(150)
    g1 = st.ifield("g").copy()
    swept = (g0 < G) & (g1 >= G)
    assert swept.sum() >= 2 * n * n                 # both boundaries moved at least one plane
    assert not np.any((g0 >= G) & (g1 < G))          # no recrystallised voxel returned to the deformed grain
    rho1 = st.field("rho").copy()
    assert np.array_equal(rho1[:, swept], mat.s_soften * rho0[:, swept])
    assert np.array_equal(rho1[:, ~swept], rho0[:, ~swept])
    k1 = st.field("k")[0]
    assert np.allclose(k1[swept], rho1[:, swept].sum(axis=0), rtol=1e-14, atol=0)
    assert ps1.X_rex == pytest.approx(ps0.X_rex + swept.sum() / N3, abs=1e-15)
    assert ps1.X_rex == pytest.approx((g1 >= G).mean(), abs=1e-15) and ps1.n_grains == 2
    st.pf_step(1)                                    # the swept voxels are recrystallised now: no second softening
    g2 = st.ifield("g")
    rho2 = st.field("rho")
    again = swept & (g2 >= G)
    assert np.array_equal(rho2[:, again], rho1[:, again])


def test_nucleation_eligibility_is_the_six_face_neighbours(mat):
    """Reading C13: a voxel is eligible when one of its six face neighbours belongs to another grain. Three
    slab bicrystals, with boundaries normal to x, y and z, nucleate wherever k > kappa is forced (kappa = 0):
    exactly the voxels on either side of each boundary, and no voxel inside a grain."""
    n = 8
    for axis in range(3):
        coord = (np.arange(n ** 3) // n ** axis) % n
        g0 = (coord >= n // 2).astype(np.int32)
        st = O.State(n, 2, g0, synth.orientations(2, 0), mat, seed=3)
        st.field("kappa")[:] = 0.0
        rc, nn = st.nucleate(0)
        grid = g0.reshape(n, n, n)                       # [z][y][x]
        gb = np.zeros_like(grid, dtype=bool)
        for ax in range(3):
            for sh in (1, -1):
                gb |= np.roll(grid, sh, axis=ax) != grid
        gb = gb.reshape(-1)
        nucleated = st.ifield("ids")[0] >= 2
        assert nn == gb.sum() == 4 * n * n
        assert np.array_equal(nucleated, gb)


def _pf_state(mat, n, G, kmax):
    g0 = np.zeros(n ** 3, dtype=np.int32)
    st = O.State(n, G, g0, synth.orientations(G, 0), mat, seed=0, kmax=kmax)
    st.field("k")[:] = 0.0
    st.ifield("ids")[:] = -1
    st.field("eta")[:] = 0.0
    st.next_id = G
    return st


def test_pf_argmax_ties_go_to_the_smaller_id(mat):
    """Reading C21: two order parameters of equal value at every point (a uniform 1/2, 1/2 mixture, which the
    step keeps exactly symmetric) give the grain id of the smaller id everywhere."""
    n = 8
    st = _pf_state(mat, n, 2, 2)
    ids, eta = st.ifield("ids"), st.field("eta")
    ids[0], ids[1] = 0, 1
    eta[0], eta[1] = 0.5, 0.5
    st.pf_step(1)
    assert np.array_equal(eta[0], eta[1])            # the tie is exact
    assert np.all(st.ifield("g") == 0)


def test_pf_active_set_keeps_the_largest_ties_to_smaller_id_and_counts_overflow(mat):
    """Reading C11 at K = 2: on the plane x = 0 of a grain-0 crystal, flanked by a plane of grain 1 (x = n-1) and
    one of grain 2 (x = 1), ids 1 and 2 arrive with exactly equal values; the point keeps its own id and the
    smaller of the tied pair, and each of those n^2 points counts once as an overflow."""
    n = 8
    st = _pf_state(mat, n, 3, 2)
    ids, eta = st.ifield("ids"), st.field("eta")
    x = np.arange(n ** 3) % n
    ids[0] = np.where(x == n - 1, 1, np.where(x == 1, 2, 0))
    eta[0] = 1.0
    rc, ps = st.pf_step(1)
    ids, eta = st.ifield("ids"), st.field("eta")
    p0 = x == 0
    assert ps.overflow == n * n and rc == 2
    assert np.all(ids[0, p0] == 0) and np.all(ids[1, p0] == 1)
    assert np.all(eta[1, p0] > mat.eta_drop)


def test_pf_drop_threshold(mat):
    """Reading C11: an order parameter leaves a point's active set when its new value falls below eta_drop
    (1e-5) and stays when it does not. A grain-0 crystal holds grain 1 at small values on two planes; the
    points next to them receive values on either side of the threshold."""
    n = 8
    st = _pf_state(mat, n, 2, 2)
    ids, eta = st.ifield("ids"), st.field("eta")
    x = np.arange(n ** 3) % n
    ids[0] = 0
    eta[0] = 1.0
    for plane, val in ((2, 3e-4), (6, 5e-5)):        # about 0.116 x val arrives next door: 3.5e-5 and 5.8e-6
        ids[1, x == plane] = 1
        eta[1, x == plane] = val
    st.pf_step(1)
    ids, eta = st.ifield("ids"), st.field("eta")
    has1 = (ids == 1).any(axis=0)
    e1 = np.where(ids == 1, eta, 0.0).sum(axis=0)
    kept = e1[has1]
    assert np.all(kept >= mat.eta_drop)              # nothing below the threshold is kept
    assert np.any((kept >= mat.eta_drop) & (kept < 10 * mat.eta_drop))   # values just above it are kept
    assert np.all(has1[(x == 1) | (x == 3)]) and not np.any(has1[(x == 5) | (x == 7)])


def test_pf_energy_nonincreasing(mat):
    n, G = 12, 6
    seeds = synth.voronoi_seeds(n, G, 8)
    g0 = O.voronoi(n, seeds)
    st = O.State(n, G, g0, synth.orientations(G, 8), mat, seed=0)
    Esc = mat.zeta * mat.mu * 1e6 * mat.b ** 2 * mat.dx / mat.omega_gb
    st.field("k")[:] = 0.5 / Esc
    ids = st.ifield("ids")
    for j, v in enumerate([5, 400, 1000, 1500]):     # four recrystallised nuclei
        ids[0, v] = G + j
    st.next_id = G + 4
    F = [st.pf_energy()]
    for _ in range(25):
        st.pf_step(1)
        F.append(st.pf_energy())
    dF = np.diff(F)
    assert np.all(dF <= 1e-9 * abs(F[0])), dF.max()
    assert F[-1] < F[0]


def test_sparse_active_set_equals_dense_bitwise(mat):
    import dataclasses
    m2 = dataclasses.replace(mat, eta_drop=-1e300)
    n, G = 8, 4
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, 4))
    a = O.State(n, G, g0, synth.orientations(G, 4), m2, seed=0, kmax=16)
    b = O.State(n, G, g0, synth.orientations(G, 4), m2, seed=0, kmax=16)
    Esc = mat.zeta * mat.mu * 1e6 * mat.b ** 2 * mat.dx / mat.omega_gb
    for s in (a, b):
        s.field("k")[:] = np.linspace(0.1, 0.6, n ** 3) / Esc
        ids = s.ifield("ids")
        ids[0, 77] = G
        ids[0, 300] = G + 1
        s.next_id = G + 2
    a.pf_step(4)
    b.pf_step_dense(4)
    assert np.array_equal(a.ifield("g"), b.ifield("g"))
    ia, ib = a.ifield("ids"), b.ifield("ids")
    ea, eb = a.field("eta"), b.field("eta")
    for v in range(n ** 3):
        da = {int(i): ea[j, v] for j, i in enumerate(ia[:, v]) if i >= 0 and ea[j, v] != 0.0}
        db = {int(i): eb[j, v] for j, i in enumerate(ib[:, v]) if i >= 0}
        assert da == db


# ------------------------------------------------------------------------------------------
# P13 gradient of the stress-strain misfit (differentiation direction)
# ------------------------------------------------------------------------------------------
def test_oracle_adjoint_gradient_matches_central_differences(mat):
    """dL/d(k1, k2, tau0, n) from the discrete adjoint equals central finite differences of the
    loss (h = 1e-6 relative) to 1e-5 relative, on a target curve the oracle makes at known
    parameters and a gradient taken at perturbed ones."""
    import dataclasses
    n, G, T, seed = 8, 4, 4, 7
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, seed))
    q = synth.orientations(G, seed)
    rc, _, _, target = O.loss_grad(n, G, g0, q, mat, seed, T, -1e-3, 1.0, want_grad=False)
    assert rc == 0
    m1 = dataclasses.replace(mat, k1=mat.k1 * 1.1, k2=mat.k2 * 0.9, tau0=mat.tau0 * 1.2, n=mat.n * 1.05)
    rc, L, g, _ = O.loss_grad(n, G, g0, q, m1, seed, T, -1e-3, 1.0, target=target)
    assert rc == 0 and L > 0
    for i, k in enumerate(("k1", "k2", "tau0", "n")):
        v = getattr(m1, k)
        h = 1e-6 * v
        Lp = O.loss_grad(n, G, g0, q, dataclasses.replace(m1, **{k: v + h}), seed, T, -1e-3, 1.0, target=target,
                         want_grad=False)[1]
        Lm = O.loss_grad(n, G, g0, q, dataclasses.replace(m1, **{k: v - h}), seed, T, -1e-3, 1.0, target=target,
                         want_grad=False)[1]
        fd = (Lp - Lm) / (2 * h)
        assert abs(g[i] / fd - 1) < 1e-5, (k, g[i], fd)


# ------------------------------------------------------------------------------------------
# augmented Lagrangian (the solver the paper names, Sec. 2.1): same fixed point as the basic scheme
# ------------------------------------------------------------------------------------------
def test_augmented_lagrangian_reaches_the_basic_scheme_solution(mat):
    n, G = 8, 5
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, 12))
    q = synth.orientations(G, 12)
    a = O.State(n, G, g0, q, mat, seed=1, tol=1e-11, max_iter=20000, scheme=0)
    b = O.State(n, G, g0, q, mat, seed=1, tol=1e-11, max_iter=20000, scheme=1, al_scale=6.0)
    for _ in range(3):
        ra, sa = a.increment(-1e-3, 1.0)
        rb, sb = b.increment(-1e-3, 1.0)
        assert ra == 0 and rb == 0
        assert sb.iterations < sa.iterations
        assert abs(sb.sig_mean[2] / sa.sig_mean[2] - 1) < 1e-9
    sig_a, sig_b = a.field("sig"), b.field("sig")
    assert np.abs(sig_a - sig_b).max() < 1e-7 * np.abs(sig_a).max()
    assert np.abs(a.field("rho") - b.field("rho")).max() < 1e-7 * a.field("rho").max()


def test_augmented_lagrangian_homogeneous_crystal_matches_point_model(mat):
    n = 4
    q = synth.orientations(1, 21)
    st = O.State(n, 1, np.zeros(n ** 3, dtype=np.int32), q, mat, seed=1, tol=1e-12, max_iter=20000, scheme=1,
                 al_scale=6.0)
    _, S, M = O.grain_tables(mat, q)
    _, hist, _ = O.point_model(mat, S[0], M[0], -1e-3, 1.0, 3)
    for inc in range(3):
        rc, s = st.increment(-1e-3, 1.0)
        assert rc == 0
        assert abs(s.sig_mean[2] / hist[inc] - 1) < 1e-9


def test_softer_reference_medium_reaches_the_same_solution_in_fewer_iterations(mat):
    """The basic scheme's fixed point does not depend on the reference medium (Moulinec-Suquet): a softer shear
    modulus mu_Voigt / 1.3, still stiffer than half of copper's largest shear stiffness C44, reaches the Voigt
    medium's converged stresses, in fewer iterations."""
    n, G = 16, 8
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, 8))
    quat = synth.orientations(G, 8)
    assert mat.mu / 1.3 > mat.C44 / 2
    out = {}
    for rs in (1.0, 1.3):
        st = O.State(n, G, g0, quat, mat, 3, tol=1e-10, newton_tol=1e-13, max_iter=4000, ref_scale=rs)
        its = []
        for _ in range(3):
            rc, s = st.increment(-1e-3, 1.0)
            assert rc == 0
            its.append(s.iterations)
        out[rs] = (st.field("sig").copy(), st.field("eps").copy(), its)
    assert np.abs(out[1.3][0] - out[1.0][0]).max() < 1e-7 * np.abs(out[1.0][0]).max()
    assert np.abs(out[1.3][1] - out[1.0][1]).max() < 1e-7 * np.abs(out[1.0][1]).max()
    assert sum(out[1.3][2]) < 0.85 * sum(out[1.0][2])


def test_oracle_state_views_outlive_their_state_and_close_safely(mat):
    """Field views keep the native oracle state alive (a view never shows freed memory), a closed state refuses
    further calls, and a state made under another build of the oracle is freed through that build."""
    import gc
    n, G = 8, 2
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, 1))
    st = O.State(n, G, g0, synth.orientations(G, 1), mat, seed=1)
    rho = st.field("rho")
    rho[0, 0] = 7.0
    del st
    gc.collect()
    for _ in range(4):      # fresh allocations that would reuse freed memory
        O.State(n, G, g0, synth.orientations(G, 1), mat, seed=2).field("rho")[:] = -1.0
    assert rho[0, 0] == 7.0 and np.all(rho[:, 1:] == mat.rho0)
    st = O.State(n, G, g0, synth.orientations(G, 1), mat, seed=1)
    st.close()
    with pytest.raises(ValueError):
        st.increment(-1e-3, 1.0)
    with O.using(O.lib()._name):
        other = O.State(n, G, g0, synth.orientations(G, 1), mat, seed=1)
    assert other._L is not O.lib()
    assert other.increment(-1e-3, 1.0)[0] == 0
    del other
    gc.collect()


def test_oracle_augmented_lagrangian_is_independent_of_the_thread_count(mat):
    """The augmented Lagrangian's stopping sums run in voxel order, so the converged state does not depend on the
    number of OpenMP threads (bitwise)."""
    n, G = 8, 4
    g0 = O.voronoi(n, synth.voronoi_seeds(n, G, 5))
    q = synth.orientations(G, 5)
    out = []
    for nt in (1, 3, os.cpu_count() or 1):
        st = O.State(n, G, g0, q, mat, seed=1, tol=1e-10, max_iter=2000, scheme=1, al_scale=6.0, nthreads=nt)
        rc, s = st.increment(-1e-3, 1.0)
        assert rc == 0
        out.append((s.iterations, st.field("sig").copy(), st.field("rho").copy()))
    for it, sig, rho in out[1:]:
        assert it == out[0][0] and np.array_equal(sig, out[0][1]) and np.array_equal(rho, out[0][2])
