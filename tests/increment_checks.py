"""Checks of a converged first increment of the power-law workload that hold at any grid size, evaluated with the
FP64 oracle: they need the fields of the solution only, so they apply to the oracle's own increments and to the
GPU's at the full size the throughput is quoted on.

- Equilibrium (Sec. 2.1): the oracle's residual sqrt(sum |xi . sigma_hat|^2) / (N^3 max(|<sigma>|, tau0)) of the
  stress field, in FP64, is within `eq_factor` x the solver tolerance.
- Mixed boundary conditions: the stress-controlled mean stresses (every Mandel slot but 33) vanish.
- At sampled voxels, the oracle's local implicit update (Eqs. HookeLaw, PlasticRate) from the total strain returns
  the stress; its shear rates give the plastic strain (dt sum_a m_a gdot_a) and the Kocks-Mecking densities from the
  uniform initial density; k is their sum. In the first increment the plastic strain at the start is zero and the
  frozen hardening is the same everywhere, tau_c = tau0 + alpha mu_Voigt b sqrt(12 rho0).
"""
import numpy as np

import oracle as O

STRESS_CONTROLLED = [0, 1, 3, 4, 5]


def check_first_increment(mat, quat, g0, n, dt, tol, fields, sig_mean_reported, sample, loc_tol, state_tol,
                          eq_factor=3.0):
    sig = np.asarray(fields["sig"], dtype=np.float64)
    out = O.stress_residual(n, sig)
    mean = out[:6]
    den = max(np.linalg.norm(mean), mat.tau0)
    err_eq = np.sqrt(out[6]) / (n ** 3 * den)
    assert err_eq <= eq_factor * tol, f"equilibrium residual {err_eq:.3e}"
    assert np.linalg.norm(mean[STRESS_CONTROLLED]) / den <= 10 * tol
    assert np.abs(mean - np.asarray(sig_mean_reported)).max() / den <= 10 * tol

    _, S, M = O.grain_tables(mat, quat)
    mu = (mat.C11 - mat.C12 + 3.0 * mat.C44) / 5.0
    tauc = mat.tau0 + mat.alpha * mu * mat.b * np.sqrt(12.0 * mat.rho0)
    eps = np.asarray(fields["eps"], dtype=np.float64)
    epsp = np.asarray(fields["epsp"], dtype=np.float64)
    rho = np.asarray(fields["rho"], dtype=np.float64)
    k = np.asarray(fields["k"], dtype=np.float64)
    want_s, want_p, want_r = [], [], []
    for v in sample:
        g = int(g0[v])
        rc, s, gd, _ = O.newton(mat, S[g], M[g], eps[:, v], tauc, dt, sig[:, v])
        assert rc >= 0, f"oracle local Newton failed at voxel {v}"
        want_s.append(s)
        want_p.append(dt * M[g].T @ gd)
        want_r.append(O.km_update(mat, np.full(12, mat.rho0), gd, dt))
    want_s, want_p, want_r = np.array(want_s).T, np.array(want_p).T, np.array(want_r).T
    smax = np.abs(sig).max()
    assert np.abs(want_s - sig[:, sample]).max() <= loc_tol * smax
    pmax = np.abs(want_p).max()
    assert pmax > 0.0
    assert np.abs(want_p - epsp[:, sample]).max() <= state_tol * pmax
    assert np.abs(want_r - rho[:, sample]).max() <= state_tol * np.abs(want_r).max()
    assert np.abs(want_r.sum(axis=0) - k[sample]).max() <= state_tol * np.abs(want_r.sum(axis=0)).max()
    return err_eq


def check_increment(mat, quat, g0, n, dt, tol, before, after, sig_mean_reported, sample, loc_tol, state_tol,
                    eq_factor=3.0):
    """The same checks for any increment of the power-law workload, from the state before it (plastic strain and
    densities) and after it (stress, total strain, plastic strain, densities, k): equilibrium and boundary
    conditions of the new stress; at sampled voxels the local implicit update from the trial strain (total strain
    after minus plastic strain before) with tau_c frozen at the densities before (reading C7), the plastic strain
    and Kocks-Mecking densities it advances, and k, their sum."""
    sig = np.asarray(after["sig"], dtype=np.float64)
    out = O.stress_residual(n, sig)
    mean = out[:6]
    den = max(np.linalg.norm(mean), mat.tau0)
    err_eq = np.sqrt(out[6]) / (n ** 3 * den)
    assert err_eq <= eq_factor * tol, f"equilibrium residual {err_eq:.3e}"
    assert np.linalg.norm(mean[STRESS_CONTROLLED]) / den <= 10 * tol
    assert np.abs(mean - np.asarray(sig_mean_reported)).max() / den <= 10 * tol
    _, S, M = O.grain_tables(mat, quat)
    mu = (mat.C11 - mat.C12 + 3.0 * mat.C44) / 5.0
    eps = np.asarray(after["eps"], dtype=np.float64)
    p0 = np.asarray(before["epsp"], dtype=np.float64)
    r0 = np.asarray(before["rho"], dtype=np.float64)
    p1 = np.asarray(after["epsp"], dtype=np.float64)
    r1 = np.asarray(after["rho"], dtype=np.float64)
    k1 = np.asarray(after["k"], dtype=np.float64)
    ws, wp, wr = [], [], []
    for v in sample:
        g = int(g0[v])
        tauc = mat.tau0 + mat.alpha * mu * mat.b * np.sqrt(r0[:, v].sum())
        rc, s, gd, _ = O.newton(mat, S[g], M[g], eps[:, v] - p0[:, v], tauc, dt, sig[:, v])
        assert rc >= 0, f"oracle local Newton failed at voxel {v}"
        ws.append(s)
        wp.append(p0[:, v] + dt * M[g].T @ gd)
        wr.append(O.km_update(mat, r0[:, v], gd, dt))
    ws, wp, wr = np.array(ws).T, np.array(wp).T, np.array(wr).T
    assert np.abs(ws - sig[:, sample]).max() <= loc_tol * np.abs(sig).max()
    assert np.abs(wp - p1[:, sample]).max() <= state_tol * np.abs(wp - p0[:, sample]).max()
    assert np.abs(wr - r1[:, sample]).max() <= state_tol * np.abs(wr - r0[:, sample]).max()
    assert np.abs(r1[:, sample].sum(axis=0) - k1[sample]).max() <= 1e-6 * np.abs(k1[sample]).max()
    return err_eq
