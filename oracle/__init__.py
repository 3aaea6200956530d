"""ctypes wrapper of the FP64 CPU oracle (liboracle.so, built from oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's CPU
baseline and reference legs (the oracle timed on the host). The product package never imports this module.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP over voxels, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", _LIB, src, "-lm"])
    return _LIB


class Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in (
        "C11", "C12", "C44", "gdot0", "n", "tau0", "alpha", "b", "k1", "k2", "rho0", "zeta",
        "kc", "q", "s_nucl", "s_soften", "omega_gb", "dx", "l_gb", "L_dt", "eta_drop",
        "T", "Q_slip", "Q_bulk", "nu_D", "poisson", "c1", "c2", "c3", "c4", "c5", "c6", "c7", "c8", "xi")]


class Config(C.Structure):
    _fields_ = [("n", C.c_int), ("grains", C.c_int), ("kmax", C.c_int), ("tol", C.c_double),
                ("max_iter", C.c_int), ("allow_unconverged", C.c_int), ("newton_tol", C.c_double),
                ("newton_max", C.c_int), ("predictor", C.c_int), ("nthreads", C.c_int), ("scheme", C.c_int),
                ("al_scale", C.c_double), ("pf_refine", C.c_int), ("law", C.c_int), ("ref_scale", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("newton_max_iters", C.c_int), ("status", C.c_int),
                ("err_eq", C.c_double), ("err_bc", C.c_double), ("sig_mean", C.c_double * 6),
                ("E", C.c_double * 6)]


class PFStats(C.Structure):
    _fields_ = [("F_tot", C.c_double), ("X_rex", C.c_double), ("n_grains", C.c_int), ("overflow", C.c_int)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_cp = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _declare(C.CDLL(_LIB))
    return _lib


@contextlib.contextmanager
def using(path):
    """Run the wrappers on another build of oracle.c (tests build copies with planted mistakes to show that the
    pins catch them); the default library is back on exit."""
    global _lib
    saved = lib()
    _lib = _declare(C.CDLL(os.path.abspath(path)))
    try:
        yield _lib
    finally:
        _lib = saved


def _declare(L):
    """ctypes signatures of every oracle entry point."""
    L.orc_mix64.restype = C.c_uint64
    L.orc_mix64.argtypes = [C.c_uint64]
    L.orc_u01.restype = C.c_double
    L.orc_u01.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.orc_weibull.restype = C.c_double
    L.orc_weibull.argtypes = [C.c_double, C.c_double, C.c_double]
    L.orc_voronoi.argtypes = [C.c_int, C.c_int, _lp, _ip]
    L.orc_quat_to_R.argtypes = [_dp, _dp]
    L.orc_slip_systems.argtypes = [_dp, _dp]
    L.orc_grain_tables.argtypes = [C.POINTER(Params), C.c_int, _dp, _dp, _dp, _dp]
    L.orc_fft1d.argtypes = [_cp, C.c_int, C.c_long, C.c_int]
    L.orc_fft3d.argtypes = [C.c_int, _cp, C.c_int]
    L.orc_dft3d_brute.argtypes = [C.c_int, _cp, _cp, C.c_int]
    L.orc_gamma0.argtypes = [_dp, C.c_double, C.c_double, _dp]
    L.orc_newton.restype = C.c_int
    L.orc_newton.argtypes = [C.POINTER(Params), _dp, _dp, _dp, C.c_double, C.c_double, C.c_double, C.c_int,
                             _dp, _dp, C.POINTER(C.c_int)]
    L.orc_residual.argtypes = [C.POINTER(Params), _dp, _dp, _dp, C.c_double, C.c_double, _dp, _dp, _dp]
    L.orc_stress_residual.argtypes = [C.c_int, _dp, _dp]
    L.orc_km_update.argtypes = [C.POINTER(Params), _dp, _dp, C.c_double]
    L.orc_point_model.restype = C.c_int
    L.orc_point_model.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                  C.c_int, _dp]
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(Config), C.POINTER(Params), _ip, _dp, C.c_uint64]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_field.restype = C.POINTER(C.c_double)
    L.orc_field.argtypes = [C.c_void_p, C.c_char_p]
    L.orc_ifield.restype = C.POINTER(C.c_int32)
    L.orc_ifield.argtypes = [C.c_void_p, C.c_char_p]
    L.orc_increment.restype = C.c_int
    L.orc_increment.argtypes = [C.c_void_p, C.c_double, C.c_double, C.POINTER(Stats)]
    L.orc_nucleate.restype = C.c_int
    L.orc_nucleate.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(C.c_int32)]
    L.orc_loss_grad.restype = C.c_int
    L.orc_loss_grad.argtypes = [C.POINTER(Config), C.POINTER(Params), _ip, _dp, C.c_uint64, C.c_int, C.c_double,
                                C.c_double, C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_void_p,
                                C.c_double]
    L.orc_pf_step.restype = C.c_int
    L.orc_pf_step.argtypes = [C.c_void_p, C.c_int, C.POINTER(PFStats)]
    L.orc_pf_step_dense.restype = C.c_int
    L.orc_pf_step_dense.argtypes = [C.c_void_p, C.c_int]
    L.orc_pf_energy.restype = C.c_double
    L.orc_pf_energy.argtypes = [C.c_void_p]
    L.orc_stats_now.argtypes = [C.c_void_p, C.POINTER(PFStats)]
    L.orc_next_id.restype = C.c_int
    L.orc_next_id.argtypes = [C.c_void_p]
    L.orc_set_next_id.argtypes = [C.c_void_p, C.c_int]
    L.orc_refresh_derived.argtypes = [C.c_void_p]
    L.orc_mr_tables.argtypes = [_dp]
    L.orc_mr_project.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_mr_frozen.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp]
    L.orc_mr_rho_m.restype = C.c_double
    L.orc_mr_rho_m.argtypes = [C.POINTER(Params), C.c_double, C.c_double]
    L.orc_mr_gdot.restype = C.c_double
    L.orc_mr_gdot.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                              C.POINTER(C.c_double)]
    L.orc_mr_ssd_rate.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double, _dp]
    L.orc_vm_stress.restype = C.c_double
    L.orc_vm_stress.argtypes = [_dp]
    L.orc_vm_strain.restype = C.c_double
    L.orc_vm_strain.argtypes = [_dp]
    L.orc_mr_grain_vectors.argtypes = [C.c_int, _dp, _dp, _dp]
    L.orc_mr_gnd_rates.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_double, C.c_double, _dp, _dp]
    L.orc_mr_gnd_rates_voxel.argtypes = [C.c_int, _ip, _ip, _dp, _dp, _dp, C.c_double, C.c_double, C.c_long,
                                         _dp, _dp]
    L.orc_mr_leff_next.restype = C.c_double
    L.orc_mr_leff_next.argtypes = [C.c_double, _dp, C.c_double]
    L.orc_newton_mr.restype = C.c_int
    L.orc_newton_mr.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                C.c_double, C.c_int, _dp, _dp, C.POINTER(C.c_int)]
    L.orc_residual_mr.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp]
    L.orc_point_model_mr.restype = C.c_int
    L.orc_point_model_mr.argtypes = [C.POINTER(Params), _dp, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                     C.c_int, _dp]
    L.orc_leff.restype = C.c_double
    L.orc_leff.argtypes = [C.c_void_p]
    return L


def make_params(mat) -> Params:
    p = Params()
    for k, _ in Params._fields_:
        setattr(p, k, float(getattr(mat, k)))
    return p


# ---------------------------------------------------------------------------------------------
# thin numpy-facing helpers
# ---------------------------------------------------------------------------------------------
def u01(seed, idx, draw):
    return lib().orc_u01(seed, idx, draw)


def weibull(u, kc, q):
    return lib().orc_weibull(u, kc, q)


def voronoi(n, seeds):
    seeds = np.ascontiguousarray(seeds, dtype=np.int64)
    out = np.zeros(n ** 3, dtype=np.int32)
    lib().orc_voronoi(n, seeds.shape[0], seeds.reshape(-1), out)
    return out


def quat_to_R(q):
    R = np.zeros(9)
    lib().orc_quat_to_R(np.ascontiguousarray(q, dtype=np.float64), R)
    return R.reshape(3, 3)


def slip_systems():
    d = np.zeros(36)
    nr = np.zeros(36)
    lib().orc_slip_systems(d, nr)
    return d.reshape(12, 3), nr.reshape(12, 3)


def grain_tables(mat, quat):
    quat = np.ascontiguousarray(quat, dtype=np.float64).reshape(-1, 4)
    G = quat.shape[0]
    Cm = np.zeros(G * 36)
    Sm = np.zeros(G * 36)
    Mm = np.zeros(G * 72)
    p = make_params(mat)
    lib().orc_grain_tables(C.byref(p), G, quat.reshape(-1), Cm, Sm, Mm)
    return Cm.reshape(G, 6, 6), Sm.reshape(G, 6, 6), Mm.reshape(G, 12, 6)


def fft3d(a, sign=-1):
    a = np.ascontiguousarray(a, dtype=np.complex128).copy()
    n = a.shape[0]
    lib().orc_fft3d(n, a.reshape(-1), sign)
    return a


def fft1d(a, sign=-1):
    a = np.ascontiguousarray(a, dtype=np.complex128).copy()
    lib().orc_fft1d(a, a.shape[0], 1, sign)
    return a


def dft3d_brute(a, sign=-1):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    out = np.zeros_like(a)
    lib().orc_dft3d_brute(a.shape[0], a.reshape(-1), out.reshape(-1), sign)
    return out


def gamma0(xi, lam0, mu0):
    G = np.zeros(36)
    lib().orc_gamma0(np.ascontiguousarray(xi, dtype=np.float64), lam0, mu0, G)
    return G.reshape(6, 6)


def newton(mat, S, M, eps_tr, tauc, dt, sig0, tol=1e-12, maxit=50):
    p = make_params(mat)
    sig = np.ascontiguousarray(sig0, dtype=np.float64).copy()
    gd = np.zeros(12)
    its = C.c_int(0)
    rc = lib().orc_newton(C.byref(p), np.ascontiguousarray(S, dtype=np.float64).reshape(-1),
                          np.ascontiguousarray(M, dtype=np.float64).reshape(-1),
                          np.ascontiguousarray(eps_tr, dtype=np.float64), tauc, dt, tol, maxit, sig, gd,
                          C.byref(its))
    return rc, sig, gd, its.value


def residual(mat, S, M, eps_tr, tauc, dt, sig):
    p = make_params(mat)
    r = np.zeros(6)
    K = np.zeros(36)
    lib().orc_residual(C.byref(p), np.ascontiguousarray(S, dtype=np.float64).reshape(-1),
                       np.ascontiguousarray(M, dtype=np.float64).reshape(-1),
                       np.ascontiguousarray(eps_tr, dtype=np.float64), tauc, dt,
                       np.ascontiguousarray(sig, dtype=np.float64), r, K)
    return r, K.reshape(6, 6)


def stress_residual(n, sig):
    """[mean stress (6), sum_xi |xi.sigma_hat|^2] of a (6, N^3) stress field."""
    out = np.zeros(7)
    lib().orc_stress_residual(n, np.ascontiguousarray(sig, dtype=np.float64).reshape(-1), out)
    return out


def km_update(mat, rho, gdot, dt):
    p = make_params(mat)
    rho = np.ascontiguousarray(rho, dtype=np.float64).copy()
    lib().orc_km_update(C.byref(p), rho, np.ascontiguousarray(gdot, dtype=np.float64), dt)
    return rho


def point_model(mat, S, M, dE33, dt, nsteps, rho0=None):
    p = make_params(mat)
    sig = np.zeros(6)
    epsp = np.zeros(6)
    rho = np.full(12, mat.rho0 if rho0 is None else rho0, dtype=np.float64)
    E = np.zeros(6)
    hist = np.zeros(max(nsteps, 1))
    rc = lib().orc_point_model(C.byref(p), np.ascontiguousarray(S, dtype=np.float64).reshape(-1),
                               np.ascontiguousarray(M, dtype=np.float64).reshape(-1), sig, epsp, rho, E,
                               dE33, dt, nsteps, hist)
    return rc, hist[:nsteps], dict(sig=sig, epsp=epsp, rho=rho, E=E)


def loss_grad(n, grains, g0, quat, mat, seed, T, dE33, dt, target=None, want_grad=True, tol=1e-12,
              max_iter=20000, adj_tol=1e-12, nthreads=0):
    """FP64 loss L = sum_t (<sigma33>_t - target_t)^2 over T increments, its adjoint gradient with
    respect to (k1, k2, tau0, n) and the stress-strain curve."""
    cfg = Config(n, grains, 8, tol, max_iter, 0, 1e-13, 60, 1, nthreads, 0, 4.0, 1, 0, 1.0)
    p = make_params(mat)
    g0 = np.ascontiguousarray(g0, dtype=np.int32).reshape(-1)
    q = np.ascontiguousarray(quat, dtype=np.float64).reshape(-1)
    tg = None if target is None else np.ascontiguousarray(target, dtype=np.float64)
    loss = C.c_double(0.0)
    grad = np.zeros(4)
    s33 = np.zeros(T)
    rc = lib().orc_loss_grad(C.byref(cfg), C.byref(p), g0, q, seed, T, dE33, dt,
                             None if tg is None else tg.ctypes.data, C.byref(loss),
                             grad.ctypes.data if want_grad else None, s33.ctypes.data, adj_tol)
    return rc, loss.value, grad, s33


class _Handle:
    """Owns one native oracle state and frees it through the library that created it, once nothing refers to it
    any more: neither its State nor any array view of its fields. A view can therefore never outlive the memory it
    shows, and a state made under one build (see using()) is never freed through another."""

    def __init__(self, L, h):
        self.L, self.h = L, h

    def __del__(self):
        h, self.h = self.h, None
        if h:
            self.L.orc_destroy(h)


class _View:
    """An array interface over native memory that holds its _Handle alive."""

    def __init__(self, owner, addr, shape, typestr):
        self._owner = owner
        self.__array_interface__ = {"data": (addr, False), "shape": tuple(shape), "typestr": typestr, "version": 3}


class State:
    """The oracle's full simulation state (FP64, host memory)."""

    def __init__(self, n, grains, g0, quat, mat, seed, kmax=8, tol=1e-10, max_iter=1000,
                 allow_unconverged=0, newton_tol=1e-12, newton_max=50, predictor=1, nthreads=0, scheme=0,
                 al_scale=4.0, pf_refine=1, law=0, ref_scale=1.0):
        self.n, self.G, self.K = n, grains, kmax
        self.N3 = n ** 3
        self.r = 2 if pf_refine == 2 else 1
        self.npf = self.r * n
        self.N3pf = self.npf ** 3
        self.mat = mat
        self._cfg = Config(n, grains, kmax, tol, max_iter, allow_unconverged, newton_tol, newton_max,
                           predictor, nthreads, scheme, al_scale, self.r, law, ref_scale)
        self.law = law
        self._p = make_params(mat)
        self._g0 = np.ascontiguousarray(g0, dtype=np.int32).reshape(-1)
        self._q = np.ascontiguousarray(quat, dtype=np.float64).reshape(-1)
        self._L = lib()      # every call on this state goes to the build that created it
        self._hd = _Handle(self._L, self._L.orc_create(C.byref(self._cfg), C.byref(self._p), self._g0, self._q,
                                                     seed))

    @property
    def h(self):
        if self._hd is None:
            raise ValueError("oracle state is closed")
        return self._hd.h

    def close(self):
        """Release the state. The native memory is freed now, or when the last field view of it goes away."""
        self._hd = None

    _SIZES = {"eps": 6, "epsp": 6, "sig": 6, "deps_prev": 6, "rho": 12, "k": 1, "kappa": 1, "gnds": 12,
              "gndet": 12, "gnd": 12}

    def _view(self, ptr, shape, typestr):
        if not ptr:
            raise ValueError("no such oracle field")
        return np.asarray(_View(self._hd, C.cast(ptr, C.c_void_p).value, shape, typestr))

    def field(self, name):
        """A view (not a copy) of a double field, shaped (components, N^3); it keeps the state alive."""
        ptr = self._L.orc_field(self.h, name.encode())
        if name in ("E", "dE_prev"):
            shape = (6,)
        elif name == "eta":   # on the phase-field grid
            shape = (self.K, self.N3pf)
        elif name == "kpf":
            shape = (self.N3pf,)
        else:
            shape = (self._SIZES[name], self.N3)
        return self._view(ptr, shape, "<f8")

    def ifield(self, name):
        ptr = self._L.orc_ifield(self.h, name.encode())
        if name == "ids":   # on the phase-field grid
            shape = (self.K, self.N3pf)
        elif name == "gpf":
            shape = (self.N3pf,)
        else:
            shape = (self.N3,)
        return self._view(ptr, shape, "<i4")

    def increment(self, dE33, dt):
        st = Stats()
        rc = self._L.orc_increment(self.h, dE33, dt, C.byref(st))
        return rc, st

    def nucleate(self, step=0):
        nn = C.c_int32(0)
        rc = self._L.orc_nucleate(self.h, step, C.byref(nn))
        return rc, nn.value

    def pf_step(self, nsteps):
        st = PFStats()
        rc = self._L.orc_pf_step(self.h, nsteps, C.byref(st))
        return rc, st

    def pf_step_dense(self, nsteps):
        return self._L.orc_pf_step_dense(self.h, nsteps)

    def pf_energy(self):
        return self._L.orc_pf_energy(self.h)

    def stats(self):
        st = PFStats()
        self._L.orc_stats_now(self.h, C.byref(st))
        return st

    @property
    def next_id(self):
        return self._L.orc_next_id(self.h)

    @next_id.setter
    def next_id(self, v):
        self._L.orc_set_next_id(self.h, int(v))

    def refresh_derived(self):
        self._L.orc_refresh_derived(self.h)

    @property
    def leff(self):
        """Effective GND length l_eff of the Ma-Roters law (Eq. L0evolution), m."""
        return self._L.orc_leff(self.h)


# ---------------------------------------------------------------------------------------------
# Ma-Roters dislocation law (Sec. 2.2)
# ---------------------------------------------------------------------------------------------
def _a(x, n=None):
    a = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    if n is not None:
        assert a.size == n
    return a


def mr_tables():
    """(|cos(n,t)|, |cos(n,d)|, |sin(n,t)|, |sin(n,d)|), each 12 x 12 [alpha, beta]."""
    t = np.zeros(576)
    lib().orc_mr_tables(t)
    return t.reshape(4, 12, 12)


def mr_project(ssd, gs=None, ge=None):
    z = np.zeros(12)
    rF, rP = np.zeros(12), np.zeros(12)
    lib().orc_mr_project(mr_tables().reshape(-1), _a(ssd, 12), _a(z if gs is None else gs, 12),
                         _a(z if ge is None else ge, 12), rF, rP)
    return rF, rP


def mr_frozen(mat, rF, rP):
    p = make_params(mat)
    tp, tcut, A = np.zeros(12), np.zeros(12), np.zeros(12)
    lib().orc_mr_frozen(C.byref(p), _a(rF, 12), _a(rP, 12), tp, tcut, A)
    return tp, tcut, A


def mr_rho_m(mat, rF, rP):
    return lib().orc_mr_rho_m(C.byref(make_params(mat)), float(rF), float(rP))


def mr_gdot(tau, tp, tcut, A):
    """(gdot, d gdot / d tau, potential) of one slip system."""
    dg, psi = C.c_double(0.0), C.c_double(0.0)
    g = lib().orc_mr_gdot(float(tau), float(tp), float(tcut), float(A), C.byref(dg), C.byref(psi))
    return g, dg.value, psi.value


def mr_ssd_rate(mat, ssd, rF, rP, tau, gd, svm, gvm):
    out = np.zeros(12)
    lib().orc_mr_ssd_rate(C.byref(make_params(mat)), _a(ssd, 12), _a(rF, 12), _a(rP, 12), _a(tau, 12),
                          _a(gd, 12), float(svm), float(gvm), out)
    return out


def vm_stress(sig):
    return lib().orc_vm_stress(_a(sig, 6))


def vm_strain(e):
    return lib().orc_vm_strain(_a(e, 6))


def mr_grain_vectors(quat):
    q = _a(quat)
    G = q.size // 4
    dv, tv = np.zeros(36 * G), np.zeros(36 * G)
    lib().orc_mr_grain_vectors(G, q, dv, tv)
    return dv.reshape(G, 12, 3), tv.reshape(G, 12, 3)


def mr_gnd_rates(n, g, g0, gd, quat, leff, b):
    """(rho_dot_GNDs, rho_dot_GNDet), each 12 x N^3, of a shear-rate field gd (12 x N^3)."""
    dv, tv = mr_grain_vectors(quat)
    N3 = n ** 3
    rs, re = np.zeros(12 * N3), np.zeros(12 * N3)
    lib().orc_mr_gnd_rates(n, np.ascontiguousarray(g, dtype=np.int32).reshape(-1),
                           np.ascontiguousarray(g0, dtype=np.int32).reshape(-1), _a(gd, 12 * N3),
                           dv.reshape(-1), tv.reshape(-1), float(leff), float(b), rs, re)
    return rs.reshape(12, N3), re.reshape(12, N3)


def mr_gnd_rates_voxel(n, g, g0, gd, quat, leff, b, v):
    """The GND rates of voxel v alone (reads gd at v and its six face neighbours only)."""
    dv, tv = mr_grain_vectors(quat)
    rs, re = np.zeros(12), np.zeros(12)
    lib().orc_mr_gnd_rates_voxel(n, np.ascontiguousarray(g, dtype=np.int32).reshape(-1),
                                 np.ascontiguousarray(g0, dtype=np.int32).reshape(-1), _a(gd, 12 * n ** 3),
                                 dv.reshape(-1), tv.reshape(-1), float(leff), float(b), int(v), rs, re)
    return rs, re


def mr_leff_next(leff, E, xi):
    return lib().orc_mr_leff_next(float(leff), _a(E, 6), float(xi))


def newton_mr(mat, S, M, eps_tr, tp, tcut, A, tref, dt, sig0, tol=1e-12, maxit=50):
    p = make_params(mat)
    sig = _a(sig0, 6).copy()
    gd = np.zeros(12)
    its = C.c_int(0)
    rc = lib().orc_newton_mr(C.byref(p), _a(S, 36), _a(M, 72), _a(eps_tr, 6), _a(tp, 12), _a(tcut, 12), _a(A, 12),
                             float(tref), float(dt), tol, maxit, sig, gd, C.byref(its))
    return rc, sig, gd, its.value


def residual_mr(mat, S, M, eps_tr, tp, tcut, A, dt, sig):
    r = np.zeros(6)
    lib().orc_residual_mr(C.byref(make_params(mat)), _a(S, 36), _a(M, 72), _a(eps_tr, 6), _a(tp, 12),
                          _a(tcut, 12), _a(A, 12), float(dt), _a(sig, 6), r)
    return r


def point_model_mr(mat, S, M, dE33, dt, nsteps, ssd0=None):
    p = make_params(mat)
    sig, epsp, E = np.zeros(6), np.zeros(6), np.zeros(6)
    ssd = np.full(12, mat.rho0 if ssd0 is None else ssd0, dtype=np.float64)
    hist = np.zeros(max(nsteps, 1))
    rc = lib().orc_point_model_mr(C.byref(p), _a(S, 36), _a(M, 72), sig, epsp, ssd, E, dE33, dt, nsteps, hist)
    return rc, hist[:nsteps], dict(sig=sig, epsp=epsp, ssd=ssd, E=E)
