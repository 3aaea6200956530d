/*
 * evp.h -- C ABI of the GB300 (sm_103a) coupled FFT-EVP / phase-field DRX hot path.
 *
 * Method: Zhao, Low, Wang, Niezgoda, "Integrated full-field dislocation-based modeling of
 * dynamic recrystallization" (arXiv:1509.04953). Section references below are to that paper.
 *
 * Conventions
 *  - Every call returns an int status: 0 = OK, > 0 = warning, < 0 = error (EVP_ERR_*).
 *    No call aborts, traps or prints. evp_last_error() gives a one-line reason.
 *  - No call allocates device memory at run time. The caller sizes one device workspace with
 *    evp_workspace_bytes() and passes it to evp_init(); it stays owned by the caller and must
 *    outlive the handle. The handle itself is a small host object freed by evp_destroy(). The
 *    only device storage the library owns is the fixed 64 KiB scratch array of
 *    evp_stress_residual_noalloc.
 *  - All device work is enqueued on the stream given to evp_init (a cudaStream_t passed as
 *    void*; NULL = legacy default stream). Calls that return host values synchronise that
 *    stream before returning.
 *  - Units: stress MPa, lengths m, densities 1/m^2, time s. Symmetric tensors are Mandel
 *    6-vectors (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12).
 *  - Fields are structure-of-arrays over the N^3 grid with linear index v = x + N*(y + N*z),
 *    component-major: component c of voxel v sits at c*N^3 + v.
 *  - N must be a power of two, 4 <= N <= 256.
 */
#ifndef EVP_GB300_H
#define EVP_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define EVP_OK 0
#define EVP_WARN_UNCONVERGED 1   /* fixed point stopped at max_iter (allow_unconverged = 1) */
#define EVP_WARN_OVERFLOW 2      /* an active set had more than kmax members; smallest dropped */
#define EVP_ERR_ARG (-1)         /* bad argument, size or pointer */
#define EVP_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define EVP_ERR_NEWTON (-3)      /* a voxel's local Newton did not converge */
#define EVP_ERR_FIXEDPOINT (-4)  /* the Green-operator fixed point did not converge */
#define EVP_ERR_NONFINITE (-5)   /* NaN or Inf in the residual reduction */
#define EVP_ERR_OOM (-6)         /* workspace smaller than evp_workspace_bytes() / id space full */

/* precision of the field arithmetic */
#define EVP_FP64 0   /* every field, FFT and solve in FP64 */
#define EVP_MIXED 1  /* FP32 fields, FFTs and phase field; FP64 factorisation of the 6x6 local Newton
                        tangent (with EVP_NEWTON_REUSE its factors are then stored and applied in FP32)
                        and FP64 macro reductions (norms, mean stress, residuals, nucleation decision) */
#define EVP_MIXED_FAST 2  /* as EVP_MIXED, but the 6x6 tangent is factorised in FP32 too */

typedef struct {
    int n;                 /* grid points per edge */
    int grains;            /* number of initial (deformed) grains G; ids 0..G-1 */
    int kmax;              /* order parameters kept per voxel, 1..8 (active set, Sec. 2.4) */
    int precision;         /* EVP_FP64 / EVP_MIXED / EVP_MIXED_FAST */
    double tol;            /* fixed-point tolerance on err_eq and err_bc */
    int max_iter;          /* fixed-point iteration cap per increment */
    int allow_unconverged; /* 1: finish an increment at max_iter with EVP_WARN_UNCONVERGED */
    double newton_tol;     /* local Newton: stop when |d sigma| <= newton_tol (|sigma| + tau_c) */
    int newton_max;        /* local Newton iteration cap */
    int predictor;         /* 1: start each increment from the previous strain-increment field */
    int max_ids;           /* capacity of the grain-id space (>= grains); 0 = grains + 8 N^3 */
    int newton_mode;       /* 0: exact Newton every fixed-point iteration; 1: keep each voxel's factored
                              tangent across iterations (21 words per voxel in the field precision) and
                              refactor only when a step stalls (same local tolerance, same result);
                              EVP_NEWTON_* */
    int scheme;            /* EVP_SCHEME_BASIC: Green-operator fixed point (Moulinec-Suquet);
                              EVP_SCHEME_AL: augmented Lagrangian (Michel-Moulinec-Suquet), the solver the
                              paper names (Sec. 2.1); same solution, fewer iterations at high contrast */
    double al_scale;       /* EVP_SCHEME_AL: reference shear modulus = Voigt mu / al_scale (bulk kept) */
    double newton_adapt;   /* 0 solves every local problem to newton_tol; eta > 0 loosens the local tolerance
                              while the fixed point is far from converged, to max(newton_tol, eta * err) with err
                              the fixed-point residual of the previous iteration (1e-2 before the first; in
                              EVP_SCHEME_AL the larger of the compatibility and multiplier residuals); the converged
                              result meets the same tolerances, with local problems solved to newton_tol */
    int pf_refine;         /* phase-field grid spacing per mechanics spacing: 0 or 1 = the same grid; 2 = the
                              2:1 refined PF grid of Sec. 2.4 ((2n)^3 PF points; the active sets, the PF argmax
                              and the interpolated driving force live there; see pf_step and drx_nucleate) */
    int law;               /* constitutive law, EVP_LAW_*: the power law with Kocks-Mecking hardening, or the
                              paper's Ma-Roters dislocation-density law (Sec. 2.2) */
    double ref_scale;      /* EVP_SCHEME_BASIC: reference medium of the Green operator and of the mixed-BC
                              correction = Voigt bulk modulus and shear modulus mu_Voigt / ref_scale (0 or 1: the
                              Voigt average). The converged solution does not depend on it; the iteration converges
                              while the reference is stiffer than half of every local stiffness (for copper up to
                              ref_scale of about 1.45), faster the softer it is. In [0.5, 4] or 0. */
} evp_config;
#define EVP_LAW_POWER 0  /* gdot = gdot0 |tau/tau_c|^n sign(tau); rho^a by storage and dynamic recovery */
#define EVP_LAW_MR 1     /* Sec. 2.2, Eqs. FlowRule, RhoForest, RhoParallel, SSDEvolution, GNDEvolution,
                            L0evolution, TotDislocationDensity, UpdateGND; constants of Table 1. Frozen per increment:
                            tau_pass = c1 mu b sqrt(rho_P), tau_cut = Q_slip sqrt(rho_F)/(c2 c3 b^2) and the prefactor
                            2 k_B T nu_D sqrt(rho_P) exp(-Q_slip/k_B T)/(c1 c3 mu b^2). After convergence the SSD
                            densities follow the four-term law (mobile density 2 k_B T sqrt(rho_P rho_F)/(c1 c2 c3 mu
                            b^3)), the GND densities the slip-rate gradients (spacing l_eff; central differences
                            inside a grain, one-sided at its boundaries), k = sum of mobile, SSD and GND densities;
                            softening (nucleation, PF sweep) scales the GND densities only. Not available with
                            EVP_NEWTON_F32_TANGENT nor with the adjoint. */
#define EVP_SCHEME_BASIC 0
#define EVP_SCHEME_AL 1
#define EVP_NEWTON_EXACT 0
#define EVP_NEWTON_REUSE 1
#define EVP_NEWTON_F32_TANGENT 2  /* EVP_FP64 only: FP64 residual, FP32 tangent and 6x6 solve (the tangent
                                     only steers the iteration; the result is fixed by the FP64 residual) */

typedef struct {
    double C11, C12, C44;        /* cubic elastic constants, MPa */
    double gdot0, n;             /* power-law flow rule gdot = gdot0 |tau/tau_c|^n sign(tau) */
    double tau0, alpha, b;       /* tau_c = tau0 + alpha mu b sqrt(sum_a rho^a), mu = Voigt average */
    double k1, k2, rho0;         /* Kocks-Mecking storage / recovery, initial density per system */
    double zeta;                 /* stored energy E = zeta mu b^2 rho_tot (Sec. 2.4) */
    double kc, q, s_nucl, s_soften; /* Weibull nucleation strength and DRX updates (Table 2) */
    double omega_gb, dx, l_gb, L_dt, eta_drop; /* phase field: energy, spacing, width (in dx),
                                                  mobility x time step, active-set drop level */
    /* EVP_LAW_MR only (Table 1; dx is its grid size l0, rho0 the initial SSD density per system) */
    double T;                    /* temperature, K */
    double Q_slip, Q_bulk;       /* activation energies of glide and of climb, J */
    double nu_D, poisson;        /* attempt frequency (1/s) and Poisson's ratio (d_dipole); the paper prints neither */
    double c1, c2, c3, c4, c5, c6, c7, c8;  /* c4, c6 in 1/m; c7 in m^5 s^(c8-1); c6 multiplies the dipole term */
    double xi;                   /* l_eff <- l_eff (1 + eps_vm / xi) after every increment */
} evp_params;

typedef struct {
    int iterations;        /* fixed-point iterations of the increment */
    int newton_max_iters;  /* largest local Newton count seen */
    int status;
    double err_eq;         /* sqrt(sum_xi |xi.sigma_hat|^2)/|sigma_hat(0)|, xi = 2 pi k/N */
    double err_bc;         /* |<sigma>_u|/|<sigma>| over the stress-controlled components */
    double sig_mean[6];    /* volume-average stress (Mandel) */
    double E[6];           /* macroscopic strain after the increment (Mandel) */
} evp_stats;

typedef struct {
    double F_tot;          /* discrete phase-field free energy (nondimensional) */
    double X_rex;          /* fraction of PF points whose grain id is recrystallised (id >= G) */
    int n_grains;          /* number of distinct grain ids present on the PF grid */
    int overflow;          /* voxel-steps whose active set was truncated to kmax */
} pf_stats;

typedef struct evp_handle evp_handle;

/* field masks for get_fields / set_fields; fields are packed in this bit order, each as
 * (components x N^3) of the type given ("T" = double in EVP_FP64, float otherwise); the phase-field
 * fields (EVP_F_IDS, EVP_F_ETA, EVP_F_GRAIN_PF) have (components x (r N)^3), r = pf_refine */
#define EVP_F_SIG   (1u << 0)   /* stress, 6 x T */
#define EVP_F_EPS   (1u << 1)   /* total strain eps = eps_e + eps_p, 6 x T (get only) */
#define EVP_F_EPSP  (1u << 2)   /* plastic strain, 6 x T */
#define EVP_F_EPSE  (1u << 3)   /* elastic strain eps - eps_p, 6 x T */
#define EVP_F_DEPS  (1u << 4)   /* strain increment of the last increment, 6 x T */
#define EVP_F_RHO   (1u << 5)   /* dislocation density per slip system, 12 x T */
#define EVP_F_K     (1u << 6)   /* rho_tot = nucleation propensity k, 1 x double */
#define EVP_F_KAPPA (1u << 7)   /* nucleation strength kappa, 1 x double */
#define EVP_F_GRAIN (1u << 8)   /* current grain id (argmax order parameter), 1 x int32 */
#define EVP_F_G0    (1u << 9)   /* initial grain id (orientation index), 1 x int32 (get only) */
#define EVP_F_DRAWS (1u << 10)  /* kappa draws so far, 1 x int32 */
#define EVP_F_IDS   (1u << 11)  /* active-set ids, kmax x int32 per PF point (slot-major, ascending ids, -1 = empty
                                   slots last) */
#define EVP_F_ETA   (1u << 12)  /* active-set order parameters, kmax x T per PF point */
#define EVP_F_GRAIN_PF (1u << 13)  /* argmax id per PF point, 1 x int32 per PF point (get only; the same as
                                      EVP_F_GRAIN when pf_refine <= 1) */
#define EVP_F_GND   (1u << 14)  /* EVP_LAW_MR only: rho_GNDs, rho_GNDet (signed) and the accumulated rho_GND,
                                   3 x 12 x T (EVP_F_RHO then holds rho_SSD) */

/* Bytes of device workspace evp_init needs for this configuration. */
int evp_workspace_bytes(const evp_config *cfg, size_t *bytes);

/* a1 + set-up (Sec. 2.1 and 3): copies the caller's host grain-id field (N^3 int32, ids in
 * 0..G-1) and G unit quaternions (w,x,y,z; rotation crystal -> sample) to the device, builds
 * the per-grain compliance and Schmid tables of the 12 FCC {111}<110> systems, sets
 * rho^a = rho0, draws kappa ~ Weibull(q, kc) per voxel from a counter-based hash of
 * (seed, voxel, draw) (Eqs. NumCrt, NuclStrengthProb) and sets one order parameter per voxel.
 * The caller keeps ownership of its host arrays and of the workspace. */
int evp_init(evp_handle **h, const evp_config *cfg, const evp_params *p, const int32_t *grain_id,
             const double *quat, uint64_t seed, void *workspace, size_t workspace_bytes,
             void *cuda_stream);

/* a2-a7 (Sec. 2.1, Eqs. HookeLaw, PlasticRate; hardening and densities Sec. 2.2): one
 * mechanical increment under mixed conditions -- E33 advances by dE33, the other mean stresses
 * are driven to zero -- solved by the Green-operator fixed point with a per-voxel implicit
 * Newton stress update, then the plastic strain, densities, tau_c and k = rho_tot are advanced.
 * With EVP_SCHEME_AL the same increment is solved by the augmented Lagrangian iteration: err_eq then
 * reports the RMS multiplier update |C0 (eps - e)| / |<lam>|, and convergence also requires the RMS
 * compatibility gap |eps - e| / |E| below tol (on-device checks as for the basic scheme).
 * out may be NULL. Returns EVP_ERR_NEWTON / EVP_ERR_FIXEDPOINT / EVP_ERR_NONFINITE without
 * advancing the state. */
int evp_increment(evp_handle *h, double dE33, double dt, evp_stats *out);

/* a8 (Sec. 2.3 with its Appendix, Eq. UpdateGND): stochastic nucleation. A voxel with a face
 * neighbour of another grain nucleates iff k > kappa; nuclei receive fresh ids in ascending
 * voxel order, a single order parameter 1 (on every PF point of the voxel: its 8 children with
 * pf_refine = 2), densities scaled by s_soften and a new kappa drawn with kc' = s_nucl kc.
 * *n_new = nuclei created. step is recorded only (draws are counted per voxel), so results depend
 * on the seed and the call history alone. */
int drx_nucleate(evp_handle *h, uint64_t step, int32_t *n_new);

/* a9-a10 (Sec. 2.4, Eqs. TotalFreeEnergy .. PFGoverning; sparse storage as cited there):
 * nsteps explicit Allen-Cahn steps of the active-set multi-grain model, grain id = argmax,
 * then densities of voxels swept from a deformed to a recrystallised grain are scaled by
 * s_soften. out may be NULL (then F_tot and the statistics are not computed).
 * With pf_refine = 2 (Sec. 2.4's 2:1 PF grid) the steps run on the (2N)^3 PF grid, lengths in
 * PF spacings dx/2: the driving force rho_tot is interpolated trilinearly (weights 3/4 and 1/4
 * between the two nearest voxel centres per axis), and a voxel's grain id is the argmax of the
 * order parameters summed over its 8 PF children (ties to the smaller id). F_tot, X_rex and
 * n_grains are taken on the PF grid. */
int pf_step(evp_handle *h, int nsteps, pf_stats *out);

/* Copy the fields in field_mask, packed in bit order, to dst (host or device memory of
 * exactly `bytes` bytes, see evp_fields_bytes). Synchronises the stream. */
int get_fields(evp_handle *h, uint32_t field_mask, void *dst, size_t bytes, int dst_is_device);
/* Overwrite state fields from src (same packing). EVP_F_EPS and EVP_F_G0 cannot be set.
 * Setting EVP_F_RHO (or EVP_F_GND) refreshes k = rho_tot. */
int set_fields(evp_handle *h, uint32_t field_mask, const void *src, size_t bytes, int src_is_device);
/* Bytes that get_fields / set_fields expect for field_mask. */
int evp_fields_bytes(const evp_handle *h, uint32_t field_mask, size_t *bytes);

/* Macroscopic scalars of the state, for checkpointing: E[6], dE_prev[6], have_prev, next_id. */
int evp_get_scalars(const evp_handle *h, double *E6, double *dE_prev6, int *have_prev, int *next_id);
int evp_set_scalars(evp_handle *h, const double *E6, const double *dE_prev6, int have_prev, int next_id);
/* Effective GND length l_eff of EVP_LAW_MR (Eq. L0evolution; m; starts at dx, advanced after every increment):
 * read it, or set it (> 0, finite; EVP_ERR_ARG otherwise) when restoring a checkpoint. */
int evp_get_leff(const evp_handle *h, double *leff);
int evp_set_leff(evp_handle *h, double leff);
/* Change the fixed-point controls after init. */
int evp_set_solver(evp_handle *h, double tol, int max_iter, int allow_unconverged);

/* ---- differentiation (the paper calibrates k1, k2, tau0, n against stress-strain curves by hand,
 * Sec. 3; this is the gradient such a calibration needs) ----
 * Discrete adjoint of recorded mechanical increments (a2-a7): for L depending on the mean stresses
 * <sigma>_t of T increments, evp_adjoint_end returns dL/d(k1, k2, tau0, n) given gbar_t = dL/d<sigma>_t.
 * The converged increments are differentiated exactly (implicit function theorem); the adjoint
 * equilibrium problem of each increment -- stiffness C_t = inverse local Newton Jacobian, the same
 * mixed macroscopic conditions -- is solved by the same Green-operator iteration. Nucleation and
 * phase-field events in between are held fixed (they must not occur between recorded increments).
 * Checkpointing: the state is stored every `checkpoint_every` increments in the caller-owned
 * adjoint workspace; the reverse sweep recomputes each segment from its checkpoint (bitwise the same
 * forward) and keeps that segment's stresses and densities. */
int evp_adjoint_workspace_bytes(const evp_config *cfg, int n_increments, int checkpoint_every, size_t *bytes);
/* Start recording from the current state: adj_ws (device, >= evp_adjoint_workspace_bytes bytes,
 * 256-byte aligned) holds checkpoints, the segment tape and the adjoint fields. */
int evp_adjoint_begin(evp_handle *h, void *adj_ws, size_t bytes, int n_increments, int checkpoint_every);
/* One recorded increment: evp_increment plus checkpointing. At most n_increments calls. */
int evp_adjoint_step(evp_handle *h, double dE33, double dt, evp_stats *out);
/* Reverse sweep over the recorded increments. gbar: host, T x 6 doubles (dL/d<sigma>_t, Mandel).
 * grad: host, 4 doubles (dL/dk1, dL/dk2, dL/dtau0, dL/dn). tol / max_iter: adjoint fixed-point
 * controls (relative residual). Restores the state of the last recorded increment on return. */
int evp_adjoint_end(evp_handle *h, const double *gbar, double *grad, double tol, int max_iter);

/* Instrumentation. Kernel launches are always counted. With profiling on (evp_set_profiling
 * (h, 1)) every kernel launch is bracketed by CUDA events on the handle's stream and its device
 * time is accumulated per kernel class. Classes: 0 newton, 1 fft_xy_r2c, 2 fft_y_fwd,
 * 3 fft_z_gamma, 4 fft_y_inv, 5 fft_xy_c2r_update, 6 reduce, 7 predictor, 8 state_update,
 * 9 nucleate, 10 pf_step, 11 pf_soften, 12 pf_stats. Classes 1 and 5 are the x passes of the forward and
 * inverse transforms; where a (field, z) plane fits one SM's shared memory (FP32 up to n = 128, FP64 up to
 * n = 64, n >= 32) the y pass runs inside them and classes 2 and 4 stay empty. ms and launches hold
 * EVP_NCLASS entries. */
#define EVP_NCLASS 13
int evp_set_profiling(evp_handle *h, int on);
/* Profile only the classes whose bits are set in mask (bit c = class c; 0 = off). The events cost a few
 * microseconds of stream time per bracketed launch, so a timing run brackets only the class it reports. */
int evp_set_profiling_mask(evp_handle *h, uint32_t mask);
/* Synchronises the handle's stream, then copies the accumulated device time (ms, host, EVP_NCLASS doubles)
 * and bracketed launch counts (launches, host, EVP_NCLASS int64) per class; either pointer may be NULL.
 * reset != 0 zeroes the totals afterwards. EVP_ERR_ARG for a NULL handle, EVP_ERR_CUDA if the stream failed. */
int evp_kernel_times(evp_handle *h, double *ms, int64_t *launches, int reset);
/* Number of the library's kernel launches on this handle since evp_init (host counter, no synchronisation).
 * EVP_ERR_ARG for a NULL handle or output pointer. */
int evp_launch_count(const evp_handle *h, int64_t *launches);
/* Running totals over all increments: local Newton iterations (one 6x6 solve each) and
 * evaluations of the residual, tangent and potential (including backtracking trials). */
int evp_newton_counts(const evp_handle *h, int64_t *solves, int64_t *evals);
/* Running total of tangent factorisations (EVP_NEWTON_REUSE; equals solves with EVP_NEWTON_EXACT). */
int evp_newton_refreshes(const evp_handle *h, int64_t *refreshes);

/* Measured throughput of this GPU's fused multiply-add pipe (the paper has no counterpart: a measurement
 * service of this library, the denominator of the local solve's pipe utilisation). precision: EVP_FP64 measures
 * FP64, the other codes FP32. Runs the library's own kernel -- 8 independent FMA chains per thread, `iters`
 * steps each, 8 CTAs of 256 threads per SM -- on cuda_stream, times it with CUDA events, synchronises, and
 * writes *tflops = 2 x FMAs / time in TFLOP/s. sink_dev: caller-owned device buffer of at least 8 bytes that the
 * kernel may write (it keeps the chains from being optimised away; its content is meaningless). Choose iters so
 * that the kernel runs for tens of milliseconds (about 3e5 for FP32, 5e3 for FP64 on a GB300). Errors:
 * EVP_ERR_ARG for a NULL pointer, iters < 1 or an unknown precision; EVP_ERR_CUDA if a CUDA call fails. */
int evp_fma_throughput(int precision, int iters, void *sink_dev, double *tflops, void *cuda_stream);

/* Frees the handle and its CUDA events. The workspace stays the caller's (the library never owns device memory);
 * work still queued on the stream must finish before the caller frees the workspace. NULL is a no-op. */
void evp_destroy(evp_handle *h);
/* Text of the most recent error or warning recorded on this handle (later successful calls do not clear it);
 * valid until the next call on the handle. For a NULL handle: "no handle". evp_init leaves a handle to read it
 * from even when it fails (release it with evp_destroy). */
const char *evp_last_error(const evp_handle *h);

/* ---- stand-alone primitives (same kernels as the increment; used for parity tests) ---- */

/* a1: periodic Voronoi grain ids. seeds: G x 3 int64 on the sub-grid [0, N*2^16)^3 (device);
 * voxel centres sit at i*2^16 + 2^15; nearest seed by exact integer squared periodic distance,
 * ties to the smaller index. ids: N^3 int32 (device). */
int evp_voronoi(int n, int grains, const int64_t *seeds_dev, int32_t *ids_dev, void *cuda_stream);

/* a3: forward 3D real-to-complex transform of `nfields` real N^3 fields (double if precision
 * == EVP_FP64, else float; device) into half spectra [field][kz][ky][kx], kx = 0..N/2
 * (interleaved complex of the same type; device). Unnormalised, exp(-2 pi i k.x/N).
 * Needs no scratch: the y and z passes run in place in out. */
int evp_rfft3d(int n, int precision, int nfields, const void *in_dev, void *out_dev, void *cuda_stream);
/* a4 residual of a given stress field (Sec. 2.1, the equilibrium check of the spectral solve):
 * forward transform of the six Mandel stress components sig_dev (6 x N^3, T, device) into
 * spec_dev (6 half spectra as evp_rfft3d, device, output), then out_dev (7 doubles, device,
 * output) = [mean stress (6), sum over all frequencies of |xi . sigma_hat|^2] with
 * xi = 2 pi k / N. scratch_dev: caller-owned device scratch of evp_residual_scratch_bytes()
 * bytes for the per-block partial sums. err_eq = sqrt(out[6]) / (N^3 |mean|). */
int evp_residual_scratch_bytes(int n, int precision, size_t *bytes);
int evp_stress_residual(int n, int precision, const void *sig_dev, void *spec_dev, void *scratch_dev,
                        double *out_dev, void *cuda_stream);

/* Allocation-free form of evp_stress_residual (the paper has no counterpart: it is a service of
 * this library). Some callers cannot allocate device memory themselves -- typically a plug-in or
 * library component whose host application owns every device allocation and does not let its
 * components call cudaMalloc -- and so cannot supply the scratch buffer evp_stress_residual asks
 * for. This entry point takes the same inputs and outputs (sig_dev, spec_dev, out_dev, all
 * caller-owned) but keeps its scratch in a fixed array inside the library: 8192 doubles (64 KiB),
 * enough for every n <= 256 in any precision, held by each GPU that loads the library until the
 * process exits. It calls no cudaMalloc, cudaFree or other allocating routine. The first call on
 * a device looks up that array's device address (with that device current) and caches it with
 * the id of the current context; a call in a new context (after a device reset, say) looks it up
 * again. Make the first call on each device, and the first after a reset, before any stream
 * capture. All calls share the one array: calls that overlap on the GPU race and must be
 * serialised by the caller (e.g. one stream). Every scratch slot a call reads is written earlier
 * in the same call, so nothing needs clearing between calls. Sizes whose partial sums would not
 * fit return EVP_ERR_ARG. */
int evp_stress_residual_noalloc(int n, int precision, const void *sig_dev, void *spec_dev, double *out_dev,
                                void *cuda_stream);

/* inverse (complex-to-real) of evp_rfft3d, unnormalised: out = N^3 * field. in is overwritten.
 * in_dev and out_dev must be 16-byte aligned (EVP_ERR_ARG otherwise). */
int evp_irfft3d(int n, int precision, int nfields, void *in_dev, void *out_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
