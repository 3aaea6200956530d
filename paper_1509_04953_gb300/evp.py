"""Thin ctypes binding of libevp_gb300.so (the C ABI declared in include/evp.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.
PyTorch provides the device workspace (caching allocator) and the stream. There is no CPU
fallback: if the library is missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libevp_gb300.so")

EVP_OK, EVP_WARN_UNCONVERGED, EVP_WARN_OVERFLOW = 0, 1, 2
EVP_ERR = {-1: "EVP_ERR_ARG", -2: "EVP_ERR_CUDA", -3: "EVP_ERR_NEWTON", -4: "EVP_ERR_FIXEDPOINT",
           -5: "EVP_ERR_NONFINITE", -6: "EVP_ERR_OOM"}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_fast": 2}

(F_SIG, F_EPS, F_EPSP, F_EPSE, F_DEPS, F_RHO, F_K, F_KAPPA, F_GRAIN, F_G0, F_DRAWS, F_IDS, F_ETA, F_GRAIN_PF,
 F_GND) = (1 << i for i in range(15))
FIELDS = {"sig": F_SIG, "eps": F_EPS, "epsp": F_EPSP, "epse": F_EPSE, "deps": F_DEPS, "rho": F_RHO, "k": F_K,
          "kappa": F_KAPPA, "g": F_GRAIN, "g0": F_G0, "draws": F_DRAWS, "ids": F_IDS, "eta": F_ETA,
          "gpf": F_GRAIN_PF, "gnd3": F_GND}
# (components, kind) with kind "T" = field precision, "f8" = double, "i4" = int32, "K" = kmax components
_FIELD_SHAPE = {"sig": (6, "T"), "eps": (6, "T"), "epsp": (6, "T"), "epse": (6, "T"), "deps": (6, "T"),
                "rho": (12, "T"), "k": (1, "f8"), "kappa": (1, "f8"), "g": (1, "i4"), "g0": (1, "i4"),
                "draws": (1, "i4"), "ids": ("K", "i4"), "eta": ("K", "T"), "gpf": (1, "i4"), "gnd3": (36, "T")}
LAWS = {"power": 0, "mr": 1}
_PF_FIELDS = ("ids", "eta", "gpf")   # on the phase-field grid ((r n)^3 points)


class EVPError(RuntimeError):
    pass


class Config(C.Structure):
    _fields_ = [("n", C.c_int), ("grains", C.c_int), ("kmax", C.c_int), ("precision", C.c_int),
                ("tol", C.c_double), ("max_iter", C.c_int), ("allow_unconverged", C.c_int),
                ("newton_tol", C.c_double), ("newton_max", C.c_int), ("predictor", C.c_int), ("max_ids", C.c_int),
                ("newton_mode", C.c_int), ("scheme", C.c_int), ("al_scale", C.c_double),
                ("newton_adapt", C.c_double), ("pf_refine", C.c_int), ("law", C.c_int), ("ref_scale", C.c_double)]


class Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in (
        "C11", "C12", "C44", "gdot0", "n", "tau0", "alpha", "b", "k1", "k2", "rho0", "zeta",
        "kc", "q", "s_nucl", "s_soften", "omega_gb", "dx", "l_gb", "L_dt", "eta_drop",
        "T", "Q_slip", "Q_bulk", "nu_D", "poisson", "c1", "c2", "c3", "c4", "c5", "c6", "c7", "c8", "xi")]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("newton_max_iters", C.c_int), ("status", C.c_int),
                ("err_eq", C.c_double), ("err_bc", C.c_double), ("sig_mean", C.c_double * 6),
                ("E", C.c_double * 6)]


class PFStats(C.Structure):
    _fields_ = [("F_tot", C.c_double), ("X_rex", C.c_double), ("n_grains", C.c_int), ("overflow", C.c_int)]


_lib = None


def load():
    """Load libevp_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise EVPError(f"{LIB_PATH} is missing: build it with paper_1509_04953_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i, d, u64, sz = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_size_t
    L.evp_workspace_bytes.argtypes = [C.POINTER(Config), C.POINTER(sz)]
    L.evp_init.argtypes = [C.POINTER(vp), C.POINTER(Config), C.POINTER(Params), vp, vp, u64, vp, sz, vp]
    L.evp_increment.argtypes = [vp, d, d, C.POINTER(Stats)]
    L.drx_nucleate.argtypes = [vp, u64, C.POINTER(C.c_int32)]
    L.pf_step.argtypes = [vp, i, C.POINTER(PFStats)]
    L.get_fields.argtypes = [vp, C.c_uint32, vp, sz, i]
    L.set_fields.argtypes = [vp, C.c_uint32, vp, sz, i]
    L.evp_fields_bytes.argtypes = [vp, C.c_uint32, C.POINTER(sz)]
    L.evp_get_scalars.argtypes = [vp, vp, vp, vp, vp]
    L.evp_set_scalars.argtypes = [vp, vp, vp, i, i]
    L.evp_set_solver.argtypes = [vp, d, i, i]
    L.evp_get_leff.argtypes = [vp, C.POINTER(d)]
    L.evp_set_leff.argtypes = [vp, d]
    L.evp_destroy.argtypes = [vp]
    L.evp_destroy.restype = None
    L.evp_last_error.argtypes = [vp]
    L.evp_last_error.restype = C.c_char_p
    L.evp_adjoint_workspace_bytes.argtypes = [C.POINTER(Config), i, i, C.POINTER(sz)]
    L.evp_adjoint_begin.argtypes = [vp, vp, sz, i, i]
    L.evp_adjoint_step.argtypes = [vp, d, d, C.POINTER(Stats)]
    L.evp_adjoint_end.argtypes = [vp, vp, vp, d, i]
    L.evp_set_profiling.argtypes = [vp, i]
    L.evp_set_profiling_mask.argtypes = [vp, C.c_uint32]
    L.evp_kernel_times.argtypes = [vp, vp, vp, i]
    L.evp_launch_count.argtypes = [vp, vp]
    L.evp_newton_counts.argtypes = [vp, vp, vp]
    L.evp_newton_refreshes.argtypes = [vp, vp]
    L.evp_voronoi.argtypes = [i, i, vp, vp, vp]
    L.evp_rfft3d.argtypes = [i, i, i, vp, vp, vp]
    L.evp_irfft3d.argtypes = [i, i, i, vp, vp, vp]
    L.evp_residual_scratch_bytes.argtypes = [i, i, C.POINTER(sz)]
    L.evp_stress_residual.argtypes = [i, i, vp, vp, vp, vp, vp]
    L.evp_stress_residual_noalloc.argtypes = [i, i, vp, vp, vp, vp]
    L.evp_fma_throughput.argtypes = [i, i, vp, C.POINTER(d), vp]
    for f in ("evp_workspace_bytes", "evp_init", "evp_increment", "drx_nucleate", "pf_step", "get_fields",
              "set_fields", "evp_fields_bytes", "evp_get_scalars", "evp_set_scalars", "evp_set_solver",
              "evp_voronoi", "evp_rfft3d", "evp_irfft3d", "evp_set_profiling", "evp_set_profiling_mask",
              "evp_kernel_times",
              "evp_launch_count", "evp_newton_counts", "evp_residual_scratch_bytes", "evp_stress_residual",
              "evp_adjoint_workspace_bytes", "evp_adjoint_begin", "evp_adjoint_step", "evp_adjoint_end",
              "evp_newton_refreshes", "evp_get_leff", "evp_set_leff", "evp_stress_residual_noalloc",
              "evp_fma_throughput"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise EVPError("no CUDA device: libevp_gb300 runs on the GPU only")
    return torch


NEWTON_MODES = {"exact": 0, "reuse": 1, "f32_tangent": 2}
SCHEMES = {"basic": 0, "al": 1}


def make_config(n, grains, precision="fp64", kmax=8, tol=1e-10, max_iter=1000, allow_unconverged=0,
                newton_tol=None, newton_max=50, predictor=1, max_ids=0, newton=None, scheme="basic",
                al_scale=6.0, newton_adapt=None, pf_refine=1, law="power", ref_scale=1.0) -> Config:
    if newton_tol is None:
        newton_tol = 1e-12 if precision == "fp64" else 1e-5
    if newton is None:
        # measured on GB300 at 128^3: tangent reuse pays where the 6x6 solve is FP64 next to an FP32
        # residual (EVP_MIXED, 1.5x); the FP64 path runs fastest with an FP32 tangent and solve under
        # its FP64 residual (1.5x, identical iterates); the all-FP32 path with the exact Newton. The FP32
        # tangent under an FP64 residual covers the power law only.
        newton = {"mixed": "reuse", "fp64": "f32_tangent", "mixed_fast": "exact"}[precision]
        if law == "mr" and newton == "f32_tangent":
            newton = "reuse"
    if newton_adapt is None:
        # the FP64 path stays the reference: every local problem solved to newton_tol
        newton_adapt = 0.0 if precision == "fp64" else 0.1
    return Config(n, grains, kmax, PRECISION[precision], tol, max_iter, allow_unconverged, newton_tol, newton_max,
                  predictor, max_ids, NEWTON_MODES[newton], SCHEMES[scheme], al_scale, newton_adapt, pf_refine,
                  LAWS[law], ref_scale)


def make_params(mat) -> Params:
    p = Params()
    for k, _ in Params._fields_:
        setattr(p, k, float(getattr(mat, k)))
    return p


def workspace_bytes(cfg: Config) -> int:
    nb = C.c_size_t(0)
    rc = load().evp_workspace_bytes(C.byref(cfg), C.byref(nb))
    if rc != 0:
        raise EVPError(f"evp_workspace_bytes: {EVP_ERR.get(rc, rc)}")
    return nb.value


class Solver:
    """One coupled FFT-EVP / phase-field simulation living on the current CUDA device."""

    def __init__(self, n, grains, grain_id, quat, mat, seed, precision="fp64", stream=None, **cfg_kw):
        torch = _torch()
        L = load()
        self.n, self.G, self.N3 = n, grains, n ** 3
        self.precision = precision
        self.cfg = make_config(n, grains, precision, **cfg_kw)
        self.K = self.cfg.kmax
        self.r = 2 if self.cfg.pf_refine == 2 else 1
        self.npf = self.r * n
        self.N3pf = self.npf ** 3
        self.dtype = np.float64 if precision == "fp64" else np.float32
        self.params = make_params(mat)
        nbytes = workspace_bytes(self.cfg)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        gid = np.ascontiguousarray(np.asarray(grain_id, dtype=np.int32).reshape(-1))
        q = np.ascontiguousarray(np.asarray(quat, dtype=np.float64).reshape(-1))
        if gid.size != self.N3 or q.size != 4 * grains:
            raise EVPError("grain_id must have N^3 entries and quat G x 4")
        self.h = C.c_void_p()
        rc = L.evp_init(C.byref(self.h), C.byref(self.cfg), C.byref(self.params), gid.ctypes.data,
                        q.ctypes.data, seed, self._ws_ptr, nbytes, self.stream.cuda_stream)
        if rc != 0:
            msg = L.evp_last_error(self.h).decode() if self.h else ""
            self.close()
            raise EVPError(f"evp_init: {EVP_ERR.get(rc, rc)}: {msg}")

    # ---- lifecycle ----
    def close(self):
        if getattr(self, "h", None) and self.h.value:
            load().evp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, name, rc):
        if rc < 0:
            raise EVPError(f"{name}: {EVP_ERR.get(rc, rc)}: {load().evp_last_error(self.h).decode()}")
        return rc

    def last_error(self) -> str:
        return load().evp_last_error(self.h).decode()

    # ---- hot path ----
    def increment(self, dE33, dt, check=True):
        st = Stats()
        rc = load().evp_increment(self.h, dE33, dt, C.byref(st))
        if check:
            self._check("evp_increment", rc)
        return rc, st

    def nucleate(self, step=0, check=True):
        nn = C.c_int32(0)
        rc = load().drx_nucleate(self.h, step, C.byref(nn))
        if check:
            self._check("drx_nucleate", rc)
        return rc, nn.value

    def pf_step(self, nsteps, stats=True, check=True):
        st = PFStats()
        rc = load().pf_step(self.h, nsteps, C.byref(st) if stats else None)
        if check:
            self._check("pf_step", rc)
        return rc, (st if stats else None)

    def set_solver(self, tol, max_iter, allow_unconverged=0):
        self._check("evp_set_solver", load().evp_set_solver(self.h, tol, max_iter, allow_unconverged))

    # ---- fields ----
    def _shape(self, name):
        comp, kind = _FIELD_SHAPE[name]
        comp = self.K if comp == "K" else comp
        dt = {"T": self.dtype, "f8": np.float64, "i4": np.int32}[kind]
        return comp, dt

    def _points(self, name):
        return self.N3pf if name in _PF_FIELDS else self.N3

    def get(self, name):
        """Copy one field to host memory as a (components, points) array (N^3 voxels, or (r N)^3 PF points
        for ids, eta and gpf)."""
        comp, dt = self._shape(name)
        out = np.empty((comp, self._points(name)), dtype=dt)
        self._check("get_fields", load().get_fields(self.h, FIELDS[name], out.ctypes.data, out.nbytes, 0))
        return out

    def get_device(self, name):
        """Copy one field into a new CUDA tensor (components, N^3)."""
        torch = _torch()
        comp, dt = self._shape(name)
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32}[dt]
        out = torch.empty((comp, self._points(name)), dtype=tdt, device="cuda")
        self._check("get_fields", load().get_fields(self.h, FIELDS[name], out.data_ptr(),
                                                     out.numel() * out.element_size(), 1))
        return out

    def set(self, name, value):
        comp, dt = self._shape(name)
        arr = np.ascontiguousarray(np.asarray(value, dtype=dt).reshape(comp, self._points(name)))
        self._check("set_fields", load().set_fields(self.h, FIELDS[name], arr.ctypes.data, arr.nbytes, 0))

    def scalars(self):
        E = (C.c_double * 6)()
        dEp = (C.c_double * 6)()
        hp = C.c_int(0)
        nid = C.c_int(0)
        self._check("evp_get_scalars", load().evp_get_scalars(self.h, E, dEp, C.byref(hp), C.byref(nid)))
        return dict(E=np.array(E[:]), dE_prev=np.array(dEp[:]), have_prev=hp.value, next_id=nid.value)

    def set_scalars(self, E, dE_prev, have_prev, next_id):
        Ea = (C.c_double * 6)(*E)
        dA = (C.c_double * 6)(*dE_prev)
        self._check("evp_set_scalars", load().evp_set_scalars(self.h, Ea, dA, int(have_prev), int(next_id)))

    @property
    def leff(self):
        """Effective GND length l_eff of the Ma-Roters law (Eq. L0evolution), m."""
        v = C.c_double(0.0)
        self._check("evp_get_leff", load().evp_get_leff(self.h, C.byref(v)))
        return v.value

    @leff.setter
    def leff(self, value):
        self._check("evp_set_leff", load().evp_set_leff(self.h, float(value)))

    def gnd(self):
        """Ma-Roters GND densities: (rho_GNDs, rho_GNDet, rho_GND), each (12, N^3)."""
        a = self.get("gnd3")
        return a[:12], a[12:24], a[24:]

    # ---- differentiation ----
    def adjoint_begin(self, n_increments, checkpoint_every):
        """Start recording increments for a reverse sweep (workspace from PyTorch)."""
        torch = _torch()
        nb = C.c_size_t(0)
        rc = load().evp_adjoint_workspace_bytes(C.byref(self.cfg), n_increments, checkpoint_every, C.byref(nb))
        if rc != 0:
            raise EVPError(f"evp_adjoint_workspace_bytes: {EVP_ERR.get(rc, rc)}")
        self.adj_ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        ptr = (self.adj_ws.data_ptr() + 255) & ~255
        self._check("evp_adjoint_begin", load().evp_adjoint_begin(self.h, ptr, nb.value, n_increments,
                                                                  checkpoint_every))
        self.adj_T = n_increments

    def adjoint_step(self, dE33, dt):
        st = Stats()
        self._check("evp_adjoint_step", load().evp_adjoint_step(self.h, dE33, dt, C.byref(st)))
        return st

    def adjoint_end(self, gbar, tol=1e-10, max_iter=20000):
        """gbar: (T, 6) dL/d<sigma>_t. Returns dL/d(k1, k2, tau0, n)."""
        g = np.ascontiguousarray(np.asarray(gbar, dtype=np.float64).reshape(-1, 6))
        grad = np.zeros(4)
        self._check("evp_adjoint_end", load().evp_adjoint_end(self.h, g.ctypes.data, grad.ctypes.data, tol, max_iter))
        return grad

    # ---- instrumentation ----
    KERNEL_CLASSES = ("newton", "fft_xy_r2c", "fft_y_fwd", "fft_z_gamma", "fft_y_inv", "fft_xy_c2r_update", "reduce",
                      "predictor", "state_update", "nucleate", "pf_step", "pf_soften", "pf_stats")

    def set_profiling(self, on=True):
        self._check("evp_set_profiling", load().evp_set_profiling(self.h, 1 if on else 0))

    def set_profiling_classes(self, names):
        """Bracket only the named kernel classes (see KERNEL_CLASSES) with CUDA events."""
        mask = 0
        for nm in names:
            mask |= 1 << self.KERNEL_CLASSES.index(nm)
        self._check("evp_set_profiling_mask", load().evp_set_profiling_mask(self.h, mask))

    def kernel_times(self, reset=False):
        ms = (C.c_double * 13)()
        n = (C.c_int64 * 13)()
        self._check("evp_kernel_times", load().evp_kernel_times(self.h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KERNEL_CLASSES)}

    def launch_count(self):
        n = C.c_int64(0)
        self._check("evp_launch_count", load().evp_launch_count(self.h, C.byref(n)))
        return n.value

    def newton_counts(self):
        """(6x6 solves, residual evaluations, tangent factorisations) so far."""
        a = C.c_int64(0)
        b = C.c_int64(0)
        c = C.c_int64(0)
        self._check("evp_newton_counts", load().evp_newton_counts(self.h, C.byref(a), C.byref(b)))
        self._check("evp_newton_refreshes", load().evp_newton_refreshes(self.h, C.byref(c)))
        return a.value, b.value, c.value

    @property
    def next_id(self):
        return self.scalars()["next_id"]


# ---- stand-alone primitives ----
def voronoi(n, seeds):
    """Periodic Voronoi grain ids (int32 CUDA tensor of N^3) from G x 3 int64 sub-grid seeds."""
    torch = _torch()
    s = torch.as_tensor(np.ascontiguousarray(seeds, dtype=np.int64)).cuda()
    out = torch.empty(n ** 3, dtype=torch.int32, device="cuda")
    rc = load().evp_voronoi(n, s.shape[0], s.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise EVPError(f"evp_voronoi: {EVP_ERR.get(rc, rc)}")
    return out


def rfft3d(x):
    """x: (nfields, N, N, N) float32/float64 CUDA tensor, indexed [f][z][y][x] ->
    (nfields, N, N, N/2+1) complex half spectra (unnormalised)."""
    torch = _torch()
    nf, n = x.shape[0], x.shape[1]
    prec = 0 if x.dtype == torch.float64 else 1
    cd = torch.complex128 if prec == 0 else torch.complex64
    out = torch.empty((nf, n, n, n // 2 + 1), dtype=cd, device="cuda")
    rc = load().evp_rfft3d(n, prec, nf, x.contiguous().data_ptr(), out.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise EVPError(f"evp_rfft3d: {EVP_ERR.get(rc, rc)}")
    return out


def irfft3d(spec):
    """Inverse of rfft3d (unnormalised: returns N^3 x field). spec is consumed (overwritten)."""
    torch = _torch()
    nf, n = spec.shape[0], spec.shape[1]
    prec = 0 if spec.dtype == torch.complex128 else 1
    rd = torch.float64 if prec == 0 else torch.float32
    out = torch.empty((nf, n, n, n), dtype=rd, device="cuda")
    rc = load().evp_irfft3d(n, prec, nf, spec.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise EVPError(f"evp_irfft3d: {EVP_ERR.get(rc, rc)}")
    return out


def fma_throughput(precision, iters=None):
    """Measured FMA-pipe throughput of the current GPU in TFLOP/s ("fp32" or "fp64"), from the library's own
    FMA-chain kernel on the current stream."""
    torch = _torch()
    code = PRECISION["fp64"] if precision == "fp64" else PRECISION["mixed"]
    if iters is None:
        iters = 5000 if precision == "fp64" else 300000
    sink = torch.empty(2, dtype=torch.float64, device="cuda")
    tf = C.c_double(0.0)
    rc = load().evp_fma_throughput(code, int(iters), sink.data_ptr(), C.byref(tf),
                                   torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise EVPError(f"evp_fma_throughput: {EVP_ERR.get(rc, rc)}")
    return tf.value


def stress_residual(sig):
    """Equilibrium residual of a (6, N, N, N) stress field on the device (float32 or float64):
    returns (spectrum, out) with out = [mean stress (6), sum |xi.sigma_hat|^2] as a CUDA tensor."""
    torch = _torch()
    n = sig.shape[1]
    prec = 0 if sig.dtype == torch.float64 else 1
    cd = torch.complex128 if prec == 0 else torch.complex64
    L = load()
    nb = C.c_size_t(0)
    if L.evp_residual_scratch_bytes(n, prec, C.byref(nb)) != 0:
        raise EVPError("evp_residual_scratch_bytes: bad size")
    scratch = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    spec = torch.empty((6, n, n, n // 2 + 1), dtype=cd, device="cuda")
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    rc = L.evp_stress_residual(n, prec, sig.contiguous().data_ptr(), spec.data_ptr(), scratch.data_ptr(),
                               out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if rc != 0:
        raise EVPError(f"evp_stress_residual: {EVP_ERR.get(rc, rc)}")
    return spec, out
