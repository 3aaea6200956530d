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
    double mr_ga;           // Ma-Roters flow rule: prefactor per unit passing stress, A = mr_ga tau_pass
    float gdot0_f, n_f, dt_f, mr_ga_f;   // FP32 copies for the FP32 path (no FP64 conversions in the kernels)
    void set_fp32() { gdot0_f = (float)gdot0; n_f = (float)n; dt_f = (float)dt; mr_ga_f = (float)mr_ga; }
};

// Ma-Roters law (Sec. 2.2): the frozen flow-rule data of every voxel, the pair (tau_pass, 1/tau_cut) of each slip
// system, pair (a, v) at words 2 (a N^3 + v) and 2 (a N^3 + v) + 1 (one 8- or 16-byte load). tpi == nullptr
// selects the power law.
template <typename TA> struct MRPtr {
    const TA *tpi;
};

// Ma-Roters constants (built on the host in FP64; FP32 copies for the FP32 path). tab: |cos| and |sin| of the
// angles between slip-plane normals and the sense vectors t = n x d (tables 0, 2) and the slip directions d
// (tables 1, 3) of every pair of systems, [k * 144 + 12 a + b]. Scalars (stress MPa, lengths m):
//   tau_pass = tp_c sqrt(rho_P), tau_cut = tcut_c sqrt(rho_F), rho_M = rm_c sqrt(rho_P rho_F),
//   d_dipole = dd_c / |tau|, climb rate = climb_c sigma_vm gdot_vm^c8 rho^2.
template <typename T> struct MRScal {
    T tp_c, tcut_c, rm_c, dd_c, climb_c, c4, c5, c6, c8, inv_b, dt, soften;
};
struct MRConst {
    double tab[576];
    float tabf[576];
    MRScal<double> d;
    MRScal<float> f;
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
// The x and y passes together: forward = fft_x_r2c then the forward y pass, inverse = the inverse y pass then
// fft_x_c2r (same contract), with bitwise the same results. Where fft_xy_fused(n, is_double) is 1 each is one
// launch over (field, z) planes held in shared memory; otherwise the two passes are launched.
int fft_xy_fused(int n, int is_double);
template <typename T>
cudaError_t fft_xy_r2c(const T *in, void *spec, int n, int nfields, cudaStream_t s, const int *skip = nullptr);
template <typename T>
cudaError_t fft_xy_c2r(const void *spec, T *out, int n, int nfields, T scale, const double *add6,
                       cudaStream_t s, const T *base = nullptr, const int *skip = nullptr);

// ---- newton.cu ----
// solve_fp64: 1 -> the 6x6 Newton system is solved in FP64 even when TA = float.
// mrp (optional): the Ma-Roters flow data; tauc then holds the stopping scale tau_ref = min_a tau_pass^a.
template <typename TA>
cudaError_t newton_field(long N3, const TA *epst, const TA *tauc, const int32_t *g0, TA *sig, const TA *Stab,
                         const TA *Mtab, MatConst mc, double tol, int maxit, int solve_fp64, int *flags,
                         cudaStream_t s,
                         const int *skip = nullptr, const TA *tol_dev = nullptr, MRPtr<TA> mrp = MRPtr<TA>{});
// Jacobian-reuse variant: fac holds 21 factor words per voxel in TA (factorised in FP64 if solve_fp64).
// Unless force_refresh, runs in two passes with the work list wl (N3 entries, count in flags[10]);
// nsm = multiprocessors, for the grid of the second pass. two_step: the first pass also takes the chord
// iteration's next two moves where they stay on its common path (same results, fewer listed voxels).
template <typename TA>
cudaError_t newton_chord_field(long N3, const TA *epst, const TA *tauc, const int32_t *g0, TA *sig, const TA *Stab,
                               const TA *Mtab, void *fac, MatConst mc, double tol, int maxit, int solve_fp64,
                               int force_refresh, int *flags, int32_t *wl, int nsm, cudaStream_t s,
                               const int *skip = nullptr,
                               const TA *tol_dev = nullptr, MRPtr<TA> mrp = MRPtr<TA>{}, int two_step = 1);
// FP64 residual / FP32 tangent Newton (FP64 path); Stabf / Mtabf are FP32 copies of the tables.
cudaError_t newton_field_df(long N3, const double *epst, const double *tauc, const int32_t *g0, double *sig,
                            const double *Stab, const double *Mtab, const float *Stabf, const float *Mtabf,
                            MatConst mc, double tol, int maxit, int *flags, cudaStream_t s,
                            const int *skip = nullptr,
                            const double *tol_dev = nullptr);
// Augmented-Lagrangian local step, grid-stride over al_grid(N3, nsm, sizeof(TA)) blocks; part: 14 doubles per
// block. al_blocks(N3) bounds the block count (for sizing).
int al_blocks(long N3);
int al_grid(long N3, int nsm, int tsize);
template <typename TA>
cudaError_t al_local(long N3, const TA *epst, const TA *epse, const TA *tauc, const int32_t *g0, TA *sig, TA *lam, TA *p,
                     const TA *Stab, const TA *Sal, const TA *Mtab, MatConst mc, double lam0, double mu0, double tol,
                     int maxit, int solve_fp64, int init, int *flags, double *part, void *fac, int refresh,
                     cudaStream_t s, int nsm, MRPtr<TA> mrp = MRPtr<TA>{});
template <typename TA>
cudaError_t predictor(long N3, const TA *epse, const TA *deps, const TA *rho, TA *epst, TA *tauc, MatConst mc,
                      double r, const double *dE6, int use_field, cudaStream_t s);
template <typename TA>
cudaError_t state_update(long N3, const TA *sig, const TA *tauc, const int32_t *g0, const TA *Mtab, TA *epst,
                         TA *epse, TA *epsp, TA *deps, TA *rho, double *k, MatConst mc, cudaStream_t s);
template <typename TA> cudaError_t total_strain(long N3, const TA *epse, const TA *epsp, TA *eps, cudaStream_t s);

// ---- mr.cu (Ma-Roters law, Sec. 2.2) ----
// Frozen hardening of an increment: projections of the densities, the pairs (tau_pass, 1/tau_cut) per system
// (layout of MRPtr) and tref = min_a tau_pass^a (the local Newton's stopping scale).
template <typename T>
cudaError_t mr_harden(long N3, const T *ssd, const T *gs, const T *ge, T *tpi, T *tref, const MRConst &c,
                      cudaStream_t s);
// After convergence: eps_p / eps_e / strain increment as state_update, and the shear rates gd (12 x N^3) with
// aux = (sigma_vm, gdot_vm) (2 x N^3) for the density update.
template <typename T>
cudaError_t mr_rates(long N3, const T *sig, const T *tpi, const int32_t *g0, const T *Mtab, const T *epst,
                     T *epse, T *epsp, T *deps, T *gd, T *aux, MatConst mc, cudaStream_t s);
// Density update: SSD (Eq. SSDEvolution), GND from the shear-rate gradients (Eq. GNDEvolution) with spacing
// leff, and k (Eq. TotDislocationDensity). vec: per grain the sample-frame d then t of the 12 systems (72 T).
template <typename T>
cudaError_t mr_update(int n, const int32_t *g, const int32_t *g0, const T *gd, const T *aux, const T *sig,
                      const T *Mtab, const T *vec, T *ssd, T *gs, T *ge, T *gnd, double *k, const MRConst &c,
                      double leff, cudaStream_t s);
// Softening (Eq. UpdateGND): GND densities of the selected voxels times c.soften, then k. mode 1: voxels with
// g >= lo (fresh nuclei); mode 2: voxels whose grain went from deformed (gprev < lo) to recrystallised
// (g >= lo); mode 0: none softened, k recomputed everywhere.
template <typename T>
cudaError_t mr_soften(long N3, int mode, const int32_t *gprev, const int32_t *g, int lo, const T *ssd, T *gs, T *ge,
                      T *gnd, double *k, const MRConst &c, cudaStream_t s);

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
// One explicit Allen-Cahn step of the active sets (ids, eta) -> (ids2, eta2), argmax ids into g. Grids of 32 points
// per edge and more take the tiled kernel, which reads the per-row slot bounds rcur of (ids, eta) and rewrites
// rdst, the bounds of (ids2, eta2) (pf_row_bounds_bytes(n) bytes each; see pf.cu); smaller grids ignore them.
long pf_row_bounds_bytes(int n);
template <typename T>
cudaError_t pf_one_step(int n, const int32_t *ids, const T *eta, int32_t *ids2, T *eta2, int32_t *g,
                        const double *k, PFConst pc, int32_t *overflow, const uint8_t *rcur, uint8_t *rdst,
                        cudaStream_t s);
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
