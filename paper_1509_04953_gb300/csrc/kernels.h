// Host-side launchers of the device kernels (internal to libevp_gb300; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace evp {

// ---- material / solver constants passed by value to the kernels ----
struct MatConst {
    double gdot0, n, dt, tau0, alpha_mu_b, k1, k2;
    double lam0, mu0;       // reference medium (Voigt isotropic average)
    int n_int;              // n if it is a small positive integer (fast power), else 0
    float gdot0_f, n_f, dt_f;   // FP32 copies for the FP32 path (no FP64 conversions in the kernels)
    void set_fp32() { gdot0_f = (float)gdot0; n_f = (float)n; dt_f = (float)dt; }
};

// ---- fft.cu ----
struct ZCtl;   // fpctl.cuh: the fixed-point control that the z pass's last block runs
enum ZMode { Z_FWD = 0, Z_INV = 1, Z_FWD_GAMMA_INV = 2, Z_FWD_RESID = 3 };
// skip (optional, device): when *skip != 0 the launched kernel returns at once (a converged fixed point
// whose remaining queued iterations are discarded). tol_dev (optional, device): the local-solve
// tolerance to use instead of tol, set on the device between iterations.
template <typename T>
cudaError_t fft_x_r2c(const T *in, void *spec, int n, int nfields, cudaStream_t s, const int *skip = nullptr);
template <typename T>
cudaError_t fft_y(void *spec, int n, int nfields, int inverse, cudaStream_t s, const int *skip = nullptr);
template <typename T>
cudaError_t fft_z(void *spec, int n, int nfields, int mode, double lam0, double mu0, double *partials,
                  double *mean6, cudaStream_t s, const int *skip = nullptr, const ZCtl *zc = nullptr);
// x-pass complex-to-real. If add6 != nullptr: out[c] = (base ? base[c] : out[c]) + scale * field + add6[c];
// else out = field.
template <typename T>
cudaError_t fft_x_c2r(const void *spec, T *out, int n, int nfields, T scale, const double *add6,
                      cudaStream_t s, const T *base = nullptr, const int *skip = nullptr);
int fft_z_blocks(int n, int is_double);

// ---- newton.cu ----
// solve_fp64: 1 -> the 6x6 Newton system is solved in FP64 even when TA = float.
template <typename TA>
cudaError_t newton_field(long N3, const TA *epst, const TA *tauc, const int32_t *g0, TA *sig, const TA *Stab,
                         const TA *Mtab, MatConst mc, double tol, int maxit, int solve_fp64, int *flags,
                         cudaStream_t s,
                         const int *skip = nullptr, const TA *tol_dev = nullptr);
// Jacobian-reuse variant: fac holds 21 factor words per voxel in TA (factorised in FP64 if solve_fp64).
// Unless force_refresh, runs in two passes with the work list wl (N3 entries, count in flags[10]);
// nsm = multiprocessors, for the grid of the second pass.
template <typename TA>
cudaError_t newton_chord_field(long N3, const TA *epst, const TA *tauc, const int32_t *g0, TA *sig, const TA *Stab,
                               const TA *Mtab, void *fac, MatConst mc, double tol, int maxit, int solve_fp64,
                               int force_refresh, int *flags, int32_t *wl, int nsm, cudaStream_t s,
                               const int *skip = nullptr,
                               const TA *tol_dev = nullptr);
// FP64 residual / FP32 tangent Newton (FP64 path); Stabf / Mtabf are FP32 copies of the tables.
cudaError_t newton_field_df(long N3, const double *epst, const double *tauc, const int32_t *g0, double *sig,
                            const double *Stab, const double *Mtab, const float *Stabf, const float *Mtabf,
                            MatConst mc, double tol, int maxit, int *flags, cudaStream_t s,
                            const int *skip = nullptr,
                            const double *tol_dev = nullptr);
// Augmented-Lagrangian local step; part: 14 doubles per block (al_blocks blocks).
int al_blocks(long N3);
template <typename TA>
cudaError_t al_local(long N3, const TA *epst, const TA *epse, const TA *tauc, const int32_t *g0, TA *sig, TA *lam, TA *p,
                     const TA *Stab, const TA *Sal, const TA *Mtab, MatConst mc, double lam0, double mu0, double tol,
                     int maxit, int solve_fp64, int init, int *flags, double *part, void *fac, int refresh,
                     cudaStream_t s);
template <typename TA>
cudaError_t predictor(long N3, const TA *epse, const TA *deps, const TA *rho, TA *epst, TA *tauc, MatConst mc,
                      double r, const double *dE6, int use_field, cudaStream_t s);
template <typename TA>
cudaError_t state_update(long N3, const TA *sig, const TA *tauc, const int32_t *g0, const TA *Mtab, TA *epst,
                         TA *epse, TA *epsp, TA *deps, TA *rho, double *k, MatConst mc, cudaStream_t s);
template <typename TA> cudaError_t total_strain(long N3, const TA *epse, const TA *epsp, TA *eps, cudaStream_t s);

// ---- adjoint.cu ----
int adj_blocks(long N3);
template <typename TA>
cudaError_t adj_prep(long N3, const int32_t *g0, const TA *Stab, const TA *Mtab, const TA *rho_prev, const TA *sig,
                     const TA *lam_ep, TA *lam_rho, TA *Ct, TA *sbar, TA *a, TA *taub, MatConst mc, const double *gb6,
                     double *part, cudaStream_t s);
template <typename TA> cudaError_t adj_tau(long N3, const TA *Ct, const TA *eb, const TA *a, TA *tau, cudaStream_t s);
template <typename TA>
cudaError_t adj_finish(long N3, const int32_t *g0, const TA *Mtab, const TA *rho_prev, const TA *sig, const TA *Ct,
                       const TA *sbar, const TA *eb, const TA *taub, TA *lam_ep, TA *lam_rho, MatConst mc, double *part,
                       cudaStream_t s);

// ---- drx.cu ----
cudaError_t voronoi(int n, int G, const int64_t *seeds, int32_t *ids, cudaStream_t s);
template <typename T>
cudaError_t drx_init(long N3, const int32_t *g0, T *rho, double *k, double *kappa, int32_t *g, int32_t *draws,
                     int32_t *ids, T *eta, int K, double rho0, double kc, double q, uint64_t seed, cudaStream_t s);
template <typename T> cudaError_t refresh_k(long N3, const T *rho, double *k, cudaStream_t s);
int nucleate_blocks(long N3);
template <typename T>
cudaError_t nucleate(int n, int r, int K, int32_t *g, double *k, double *kappa, T *rho, int32_t *draws,
                     int32_t *ids, T *eta, int32_t *gpf, int32_t *blk_counts, int32_t *blk_offsets,
                     int32_t *count_out, int next_id, double s_soften, double kc_new, double q, uint64_t seed,
                     cudaStream_t s);

// ---- pf.cu ----
struct PFConst {
    double m, kappa, gam, L_dt, Escale, drop;
    int G, K;
    float m_f, kappa_f, gam_f, L_dt_f, drop_f;   // FP32 copies for the FP32 path
    void set_fp32() { m_f = (float)m; kappa_f = (float)kappa; gam_f = (float)gam; L_dt_f = (float)L_dt; drop_f = (float)drop; }
};
template <typename T>
cudaError_t pf_one_step(int n, const int32_t *ids, const T *eta, int32_t *ids2, T *eta2, int32_t *g,
                        const double *k, PFConst pc, int32_t *overflow, cudaStream_t s);
template <typename T>
cudaError_t pf_soften(long N3, const int32_t *gprev, const int32_t *g, T *rho, double *k, int G, double s_soften,
                      cudaStream_t s);
int pf_stat_blocks(long N3);
// 2:1 PF grid (Sec. 2.4): kpf[(2n)^3] = trilinear interpolation of k[n^3]; g[n^3] = argmax of the order
// parameters summed over each voxel's 8 PF children; initial PF active sets from the parent grain.
cudaError_t pf_interp(int n, const double *k, double *kpf, cudaStream_t s);
template <typename T>
cudaError_t pf_restrict(int n, int K, const int32_t *ids, const T *eta, int32_t *g, cudaStream_t s);
cudaError_t pf_init(int n, int r, int K, const int32_t *g0, int32_t *ids, void *eta, int32_t *ids2, void *eta2,
                    int eta_double, int32_t *gpf, cudaStream_t s);
template <typename T>
cudaError_t pf_stats_launch(int n, const int32_t *ids, const T *eta, const int32_t *g, const double *k, PFConst pc,
                     uint32_t *bitmap, int bitmap_words, double *partials, cudaStream_t s);
cudaError_t reduce_partials(const double *partials, int nparts, int nvals, double *out, cudaStream_t s,
                            const int *skip = nullptr);

}  // namespace evp
