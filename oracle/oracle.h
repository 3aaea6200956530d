/*
 * FP64 CPU oracle for the coupled FFT-EVP / phase-field DRX hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline and reference legs (the oracle timed on the host) may load this library. The product path (paper_1509_04953_gb300) never
 * includes, links or calls it, and it shares no code with that path.
 *
 * Units: stress MPa, lengths m, densities 1/m^2, time s. Symmetric tensors are Mandel
 * 6-vectors (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12). Fields are indexed
 * v = x + N*(y + N*z), component-major: f[c*N^3 + v].
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>
#include <complex.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double C11, C12, C44;      /* cubic elastic constants, MPa */
    double gdot0, n;           /* power-law flow rule */
    double tau0, alpha, b;     /* tau_c = tau0 + alpha*mu*b*sqrt(sum rho) */
    double k1, k2, rho0;       /* Kocks-Mecking storage / recovery, initial density per system */
    double zeta;               /* stored energy = zeta*mu*b^2*rho_tot */
    double kc, q, s_nucl, s_soften;
    double omega_gb, dx, l_gb, L_dt, eta_drop;
    /* Ma-Roters dislocation law (law = 1, Sec. 2.2, Table 1); dx is the grid size l0 */
    double T;                  /* temperature, K */
    double Q_slip, Q_bulk;     /* activation energies for glide and for climb, J */
    double nu_D, poisson;      /* attempt frequency, 1/s; Poisson's ratio (d_dipole) */
    double c1, c2, c3, c4, c5, c6, c7, c8;
    double xi;                 /* effective GND length: l_eff <- l_eff (1 + eps_vm / xi) */
} orc_params;

typedef struct {
    int n, grains, kmax;
    double tol;                /* fixed-point tolerance on err_eq and err_bc */
    int max_iter;
    int allow_unconverged;     /* 1: finish the increment after max_iter with a warning */
    double newton_tol;
    int newton_max;
    int predictor;             /* 1: extrapolate the previous strain-increment field */
    int nthreads;              /* OpenMP threads for per-voxel loops (0 = default) */
    int scheme;                /* 0: basic Green-operator iteration, 1: augmented Lagrangian */
    double al_scale;           /* augmented Lagrangian: reference shear modulus = mu_Voigt / al_scale */
    int pf_refine;             /* phase-field grid per mechanics grid spacing: 1 (same grid) or 2 (Sec. 2.4) */
    int law;                   /* 0: power law + Kocks-Mecking; 1: Ma-Roters dislocation law (Sec. 2.2) */
    double ref_scale;          /* basic scheme: reference shear modulus mu_Voigt / ref_scale, bulk kept (0 or 1: Voigt) */
} orc_config;

typedef struct {
    int iterations, newton_max_iters, status;
    double err_eq, err_bc;
    double sig_mean[6], E[6];
} orc_stats;

typedef struct {
    double F_tot, X_rex;
    int n_grains, overflow;
} orc_pf_stats;

typedef struct orc_state orc_state;

/* ---- primitives (pinned individually by tests/test_oracle_pins.py) ---- */
uint64_t orc_mix64(uint64_t z);
double orc_u01(uint64_t seed, uint64_t idx, uint64_t draw);
double orc_weibull(double u, double kc, double q);
void orc_voronoi(int n, int G, const int64_t *seeds, int32_t *ids);
void orc_quat_to_R(const double q[4], double R[9]);
void orc_slip_systems(double d[12][3], double nrm[12][3]);
void orc_grain_tables(const orc_params *p, int G, const double *quat, double *C, double *S, double *M);
void orc_fft1d(double complex *a, int n, long stride, int sign);
void orc_fft3d(int n, double complex *a, int sign);
void orc_dft3d_brute(int n, const double complex *in, double complex *out, int sign);
void orc_gamma0(const double xi[3], double lam0, double mu0, double G[36]);
int orc_newton(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
               double tauc, double dt, double tol, int maxit, double sig[6], double gdot[12], int *iters);
void orc_residual(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                  double tauc, double dt, const double sig[6], double r[6], double K[36]);
void orc_km_update(const orc_params *p, double *rho, const double *gdot, double dt);
int orc_point_model(const orc_params *p, const double *S, const double *M, double *sig, double *epsp,
                    double *rho, double *E, double dE33, double dt, int nsteps, double *sig33_hist);

void orc_stress_residual(int n, const double *sig, double out[7]);

/* ---- Ma-Roters dislocation law (Sec. 2.2), pinned by tests/test_oracle_mr.py ---- */
void orc_mr_tables(double tab[576]);
void orc_mr_project(const double tab[576], const double ssd[12], const double gs[12], const double ge[12],
                    double rF[12], double rP[12]);
void orc_mr_frozen(const orc_params *p, const double rF[12], const double rP[12], double tp[12], double tcut[12],
                   double A[12]);
double orc_mr_rho_m(const orc_params *p, double rF, double rP);
double orc_mr_gdot(double tau, double tp, double tcut, double A, double *dg, double *psi);
void orc_mr_ssd_rate(const orc_params *p, const double ssd[12], const double rF[12], const double rP[12],
                     const double tau[12], const double gd[12], double svm, double gvm, double rate[12]);
double orc_vm_stress(const double sig[6]);
double orc_vm_strain(const double e[6]);
void orc_mr_grain_vectors(int G, const double *quat, double *dv, double *tv);
void orc_mr_gnd_rates(int n, const int32_t *g, const int32_t *g0, const double *gd, const double *dv,
                      const double *tv, double leff, double b, double *rs, double *re);
void orc_mr_gnd_rates_voxel(int n, const int32_t *g, const int32_t *g0, const double *gd, const double *dv,
                            const double *tv, double leff, double b, long v, double rs[12], double re[12]);
double orc_mr_leff_next(double leff, const double E[6], double xi);
int orc_newton_mr(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                  const double tp[12], const double tcut[12], const double A[12], double tref, double dt,
                  double tol, int maxit, double sig[6], double gdot[12], int *iters);
void orc_residual_mr(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                     const double tp[12], const double tcut[12], const double A[12], double dt,
                     const double sig[6], double r[6]);
int orc_point_model_mr(const orc_params *p, const double *S, const double *M, double *sig, double *epsp,
                       double *ssd, double *E, double dE33, double dt, int nsteps, double *sig33_hist);
double orc_leff(orc_state *s);

/* ---- full state ---- */
orc_state *orc_create(const orc_config *cfg, const orc_params *p, const int32_t *g0, const double *quat,
                      uint64_t seed);
void orc_destroy(orc_state *s);
double *orc_field(orc_state *s, const char *name);
int32_t *orc_ifield(orc_state *s, const char *name);
int orc_increment(orc_state *s, double dE33, double dt, orc_stats *out);
int orc_nucleate(orc_state *s, uint64_t step, int32_t *n_new);
int orc_loss_grad(const orc_config *cfg, const orc_params *p, const int32_t *g0, const double *quat, uint64_t seed,
                  int T, double dE33, double dt, const double *target, double *loss, double grad[4], double *sig33,
                  double adj_tol);
int orc_pf_step(orc_state *s, int nsteps, orc_pf_stats *out);
int orc_pf_step_dense(orc_state *s, int nsteps);
double orc_pf_energy(orc_state *s);
void orc_stats_now(orc_state *s, orc_pf_stats *out);
int orc_next_id(orc_state *s);
void orc_set_next_id(orc_state *s, int next_id);
void orc_refresh_derived(orc_state *s);

#ifdef __cplusplus
}
#endif
#endif
