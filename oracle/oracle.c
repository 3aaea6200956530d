/*
 * FP64 CPU oracle of the coupled FFT-EVP / phase-field DRX hot path
 * (Zhao, Low, Wang, Niezgoda, arXiv:1509.04953).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the CPU baseline
 * and reference legs of bench.py (the oracle timed on the host). It is plain, slow and written to be checked against the paper by eye:
 * plain loops, a textbook radix-2 FFT, full 4th-order tensors, no fusion and no blocking.
 * It shares no code with the CUDA library.
 *
 * Every function names the passage of the paper (or the textbook closed form) it follows.
 * Readings of passages the paper leaves open are listed where they are used.
 *
 * Pins: each step is checked against closed forms, brute force, invariants or the paper's
 * relations by the tests. The coupled trajectory as a whole (increments, nucleation and
 * phase-field steps in sequence) is parity unpinned beyond the pins of its steps.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* complex.h defines I as the imaginary unit; the oracle uses I as a Mandel index instead */
#undef I
#define IU _Complex_I
#define SQ2 1.41421356237309504880
#define PI 3.14159265358979323846

/* Mandel index -> tensor index pair, and the Mandel weight of each slot. */
static const int MI[6] = {0, 1, 2, 1, 0, 0};
static const int MJ[6] = {0, 1, 2, 2, 2, 1};
static double mw(int I) { return I < 3 ? 1.0 : SQ2; }

/* ------------------------------------------------------------------------------------------
 * Counter-based generator: SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014), applied
 * to (seed, voxel index, draw number). u lies strictly inside (0,1).
 * ---------------------------------------------------------------------------------------- */
uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double orc_u01(uint64_t seed, uint64_t idx, uint64_t draw) {
    const uint64_t golden = 0x9E3779B97F4A7C15ULL;
    uint64_t h = orc_mix64(seed ^ 0xD1B54A32D192ED03ULL);
    h = orc_mix64(h + golden * (idx + 1));
    h = orc_mix64(h + golden * (draw + 1));
    return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Inverse of the Weibull CDF P(kappa < k) = 1 - exp(-(k/kc)^q)  (Eqs. NumCrt, NuclStrengthProb). */
double orc_weibull(double u, double kc, double q) {
    return kc * pow(-log(1.0 - u), 1.0 / q);
}

/* ------------------------------------------------------------------------------------------
 * Microstructure: periodic Voronoi tessellation. Voxel centres sit at (i*2^16 + 2^15) on the
 * integer sub-grid; a voxel joins the seed at the smallest squared periodic distance, ties
 * going to the smaller seed index. Exact integer arithmetic.
 * ---------------------------------------------------------------------------------------- */
void orc_voronoi(int n, int G, const int64_t *seeds, int32_t *ids) {
    const int64_t L = (int64_t)n << 16;
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                int64_t c[3] = {((int64_t)x << 16) + 32768, ((int64_t)y << 16) + 32768,
                                ((int64_t)z << 16) + 32768};
                int64_t best = -1;
                int arg = 0;
                for (int g = 0; g < G; ++g) {
                    int64_t d2 = 0;
                    for (int a = 0; a < 3; ++a) {
                        int64_t d = c[a] - seeds[3 * g + a];
                        if (d < 0) d = -d;
                        d %= L;
                        if (L - d < d) d = L - d;
                        d2 += d * d;
                    }
                    if (best < 0 || d2 < best) { best = d2; arg = g; }
                }
                ids[x + (size_t)n * (y + (size_t)n * z)] = arg;
            }
}

/* Rotation matrix of a unit quaternion (w,x,y,z); R maps crystal coordinates to sample ones. */
void orc_quat_to_R(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double s = 1.0 / sqrt(w * w + x * x + y * y + z * z);
    w *= s; x *= s; y *= s; z *= s;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* The 12 FCC {111}<110> slip systems (crystal frame, unit vectors): "single-phase FCC",
 * Sec. 2.2. Slip plane normals (111), (-111), (1-11), (11-1), three <110> directions each. */
void orc_slip_systems(double d[12][3], double nrm[12][3]) {
    static const double N4[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
    static const double D4[4][3][3] = {
        {{0, 1, -1}, {1, 0, -1}, {1, -1, 0}},
        {{0, 1, -1}, {1, 0, 1}, {1, 1, 0}},
        {{0, 1, 1}, {1, 0, -1}, {1, 1, 0}},
        {{0, 1, 1}, {1, 0, 1}, {1, -1, 0}}};
    for (int p = 0; p < 4; ++p)
        for (int j = 0; j < 3; ++j) {
            int a = 3 * p + j;
            for (int c = 0; c < 3; ++c) {
                nrm[a][c] = N4[p][c] / sqrt(3.0);
                d[a][c] = D4[p][j][c] / sqrt(2.0);
            }
        }
}

/* Plain Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix. */
static int inv_gj(int n, const double *A, double *Ainv) {
    double W[6][12];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) W[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(W[r][c]) > fabs(W[p][c])) p = r;
        if (W[p][c] == 0.0) return -1;
        if (p != c)
            for (int j = 0; j < 2 * n; ++j) { double t = W[c][j]; W[c][j] = W[p][j]; W[p][j] = t; }
        double piv = W[c][c];
        for (int j = 0; j < 2 * n; ++j) W[c][j] /= piv;
        for (int r = 0; r < n; ++r)
            if (r != c) {
                double f = W[r][c];
                for (int j = 0; j < 2 * n; ++j) W[r][j] -= f * W[c][j];
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = W[i][j + n];
    return 0;
}

/* Per-grain tables in the sample frame: stiffness C (Mandel 6x6), compliance S = C^-1 and
 * Schmid tensors m^a = sym(d^a x n^a) as Mandel 6-vectors (Eqs. HookeLaw, PlasticRate).
 * The cubic stiffness is rotated index by index: C'_ijkl = R_ia R_jb R_kc R_ld C_abcd. */
void orc_grain_tables(const orc_params *p, int G, const double *quat, double *C, double *S, double *M) {
    double d[12][3], nr[12][3];
    orc_slip_systems(d, nr);
    double Cc[3][3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double v = p->C12 * (i == j) * (k == l) + p->C44 * ((i == k) * (j == l) + (i == l) * (j == k));
                    if (i == j && j == k && k == l) v += p->C11 - p->C12 - 2.0 * p->C44;
                    Cc[i][j][k][l] = v;
                }
    for (int g = 0; g < G; ++g) {
        double R[9];
        orc_quat_to_R(quat + 4 * g, R);
        double Cs[3][3][3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        double acc = 0.0;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b)
                                for (int c = 0; c < 3; ++c)
                                    for (int e = 0; e < 3; ++e)
                                        acc += R[3 * i + a] * R[3 * j + b] * R[3 * k + c] * R[3 * l + e] * Cc[a][b][c][e];
                        Cs[i][j][k][l] = acc;
                    }
        double *Cg = C + 36 * g;
        for (int I = 0; I < 6; ++I)
            for (int J = 0; J < 6; ++J) Cg[6 * I + J] = mw(I) * mw(J) * Cs[MI[I]][MJ[I]][MI[J]][MJ[J]];
        inv_gj(6, Cg, S + 36 * g);
        for (int a = 0; a < 12; ++a) {
            double ds[3], ns[3];
            for (int i = 0; i < 3; ++i) {
                ds[i] = R[3 * i] * d[a][0] + R[3 * i + 1] * d[a][1] + R[3 * i + 2] * d[a][2];
                ns[i] = R[3 * i] * nr[a][0] + R[3 * i + 1] * nr[a][1] + R[3 * i + 2] * nr[a][2];
            }
            for (int I = 0; I < 6; ++I) {
                int i = MI[I], j = MJ[I];
                M[72 * g + 6 * a + I] = mw(I) * 0.5 * (ds[i] * ns[j] + ds[j] * ns[i]);
            }
        }
    }
}

/* ------------------------------------------------------------------------------------------
 * Textbook iterative radix-2 Cooley-Tukey FFT (bit reversal, then butterflies), unnormalised,
 * a[j] <- sum_k a[k] exp(sign*2*pi*i*j*k/n). n must be a power of two.
 * ---------------------------------------------------------------------------------------- */
void orc_fft1d(double complex *a, int n, long stride, int sign) {
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { double complex t = a[i * stride]; a[i * stride] = a[j * stride]; a[j * stride] = t; }
    }
    for (int len = 2; len <= n; len <<= 1)
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                double complex w = cexp(sign * 2.0 * PI * IU * (double)k / (double)len);
                double complex u = a[(i + k) * stride], v = w * a[(i + k + len / 2) * stride];
                a[(i + k) * stride] = u + v;
                a[(i + k + len / 2) * stride] = u - v;
            }
}

void orc_fft3d(int n, double complex *a, int sign) {
    const long n2 = (long)n * n;
#pragma omp parallel for schedule(static)
    for (long l = 0; l < n2; ++l) orc_fft1d(a + l * n, n, 1, sign);                 /* x lines */
#pragma omp parallel for schedule(static)
    for (long l = 0; l < n2; ++l) orc_fft1d(a + (l / n) * n2 + (l % n), n, n, sign); /* y lines */
#pragma omp parallel for schedule(static)
    for (long l = 0; l < n2; ++l) orc_fft1d(a + l, n, n2, sign);                    /* z lines */
}

/* Brute-force O(N^6) DFT, the definition written out (pins the FFT). */
void orc_dft3d_brute(int n, const double complex *in, double complex *out, int sign) {
    for (int kz = 0; kz < n; ++kz)
        for (int ky = 0; ky < n; ++ky)
            for (int kx = 0; kx < n; ++kx) {
                double complex acc = 0;
                for (int z = 0; z < n; ++z)
                    for (int y = 0; y < n; ++y)
                        for (int x = 0; x < n; ++x) {
                            long ph = ((long)kx * x + (long)ky * y + (long)kz * z) % n;
                            acc += in[x + n * (y + n * z)] * cexp(sign * 2.0 * PI * IU * (double)ph / (double)n);
                        }
                out[kx + n * (ky + n * kz)] = acc;
            }
}

/* ------------------------------------------------------------------------------------------
 * Green operator of an isotropic reference medium (lambda0, mu0) in Fourier space
 * (Moulinec-Suquet form, cited by the paper in Sec. 2.1):
 *   G_khij = [d_ki x_h x_j + d_hi x_k x_j + d_kj x_h x_i + d_hj x_k x_i] / (4 mu0 |x|^2)
 *          - (lambda0+mu0)/(mu0 (lambda0+2 mu0)) x_i x_j x_k x_h / |x|^4,
 * assembled as a full 4th-order tensor and then written in Mandel form. xi != 0.
 * ---------------------------------------------------------------------------------------- */
void orc_gamma0(const double xi[3], double lam0, double mu0, double Gm[36]) {
    double x2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    double c2 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));
    double Gt[3][3][3][3];
    for (int k = 0; k < 3; ++k)
        for (int h = 0; h < 3; ++h)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    Gt[k][h][i][j] = ((k == i) * xi[h] * xi[j] + (h == i) * xi[k] * xi[j] + (k == j) * xi[h] * xi[i] +
                                      (h == j) * xi[k] * xi[i]) / (4.0 * mu0 * x2) -
                                     c2 * xi[i] * xi[j] * xi[k] * xi[h] / (x2 * x2);
    /* Mandel form of the map sigma -> eps: eps_kh = sum_ij G_khij sigma_ij, where the
     * symmetric sum over (i,j) counts both off-diagonal slots. */
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) {
            int k = MI[I], h = MJ[I], i = MI[J], j = MJ[J];
            double v = (i == j) ? Gt[k][h][i][j] : (Gt[k][h][i][j] + Gt[k][h][j][i]);
            Gm[6 * I + J] = mw(I) * v / mw(J);
        }
}

/* ------------------------------------------------------------------------------------------
 * Constitutive law (readings of Sec. 2.2 for the power-law / Kocks-Mecking form):
 *   gdot^a = gdot0 |tau^a/tau_c|^n sign(tau^a),  tau^a = m^a : sigma.
 * Implicit Euler stress update (Eq. HookeLaw with Eq. PlasticRate), written as the strain
 * residual  r(sigma) = S:sigma + dt * sum_a m^a gdot^a(sigma) - (eps - eps_p^t) = 0.
 * r is the gradient of the convex potential
 *   Phi(sigma) = 1/2 sigma:S:sigma - sigma:eps_tr + dt sum_a gdot0 tau_c |tau^a/tau_c|^(n+1)/(n+1),
 * whose Hessian K = S + dt sum_a (n gdot0 |x^a|^(n-1)/tau_c) m^a (x) m^a is symmetric positive
 * definite. Newton steps on r with Armijo backtracking on Phi converge from any start.
 * ---------------------------------------------------------------------------------------- */
typedef struct { double r[6], K[36], phi, gdot[12]; } nt_eval;

/* Flow-rule data of one voxel, frozen over an increment: the power law's tau_c, or the Ma-Roters
 * passing stress tp, cutting stress tcut and prefactor A of every slip system (law = 1). tauc is
 * also the stress added to |sigma| in the Newton stopping scale. */
typedef struct {
    int law;
    double tauc;
    const double *tp, *tcut, *A;
} nt_flow;

static void nt_evaluate(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                        const nt_flow *f, double dt, const double sig[6], nt_eval *e) {
    const double tauc = f->tauc;
    for (int I = 0; I < 6; ++I) {
        double acc = 0.0;
        for (int J = 0; J < 6; ++J) acc += S[6 * I + J] * sig[J];
        e->r[I] = acc - eps_tr[I];
        for (int J = 0; J < 6; ++J) e->K[6 * I + J] = S[6 * I + J];
    }
    double phi = 0.0;
    for (int I = 0; I < 6; ++I) {
        double Ss = 0.0;
        for (int J = 0; J < 6; ++J) Ss += S[6 * I + J] * sig[J];
        phi += 0.5 * sig[I] * Ss - sig[I] * eps_tr[I];
    }
    for (int a = 0; a < 12; ++a) {
        const double *m = M + 6 * a;
        double tau = 0.0;
        for (int I = 0; I < 6; ++I) tau += m[I] * sig[I];
        double gd, slope;
        if (f->law == 1) {
            double dg, psi;
            gd = orc_mr_gdot(tau, f->tp[a], f->tcut[a], f->A[a], &dg, &psi);
            slope = dt * dg;
            phi += dt * psi;
        } else {
            double x = tau / tauc, ax = fabs(x);
            double pw = ax > 0.0 ? pow(ax, p->n) : 0.0;
            gd = p->gdot0 * pw * (x < 0.0 ? -1.0 : 1.0);
            if (ax == 0.0) gd = 0.0;
            slope = ax > 0.0 ? dt * p->n * p->gdot0 * (pw / ax) / tauc : 0.0;
            phi += dt * p->gdot0 * tauc * pw * ax / (p->n + 1.0);
        }
        e->gdot[a] = gd;
        for (int I = 0; I < 6; ++I) {
            e->r[I] += dt * m[I] * gd;
            for (int J = 0; J < 6; ++J) e->K[6 * I + J] += slope * m[I] * m[J];
        }
    }
    e->phi = phi;
}

void orc_residual(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                  double tauc, double dt, const double sig[6], double r[6], double K[36]) {
    nt_eval e;
    nt_flow f = {0, tauc, NULL, NULL, NULL};
    nt_evaluate(p, S, M, eps_tr, &f, dt, sig, &e);
    memcpy(r, e.r, sizeof e.r);
    memcpy(K, e.K, sizeof e.K);
}

/* Damped Newton on r(sigma) = 0 with Armijo backtracking on the convex potential whose gradient
 * is r; stops when the step is below tol (|sigma| + tau_c). */
static int nt_newton(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                     const nt_flow *f, double dt, double tol, int maxit, double sig[6], double gdot[12], int *iters) {
    nt_eval e, t;
    const double tauc = f->tauc;
    nt_evaluate(p, S, M, eps_tr, f, dt, sig, &e);
    for (int it = 1; it <= maxit; ++it) {
        double Ki[36], d[6];
        if (inv_gj(6, e.K, Ki) != 0) { *iters = it; return -1; }
        for (int I = 0; I < 6; ++I) {
            d[I] = 0.0;
            for (int J = 0; J < 6; ++J) d[I] += Ki[6 * I + J] * e.r[J];
        }
        double rd = 0.0, dn = 0.0, sn = 0.0;
        for (int I = 0; I < 6; ++I) { rd += e.r[I] * d[I]; dn += d[I] * d[I]; sn += sig[I] * sig[I]; }
        dn = sqrt(dn);
        double scale = sqrt(sn) + tauc;
        double s = 1.0, trial[6];
        int ok = 0;
        for (int h = 0; h < 60; ++h) {
            for (int I = 0; I < 6; ++I) trial[I] = sig[I] - s * d[I];
            nt_evaluate(p, S, M, eps_tr, f, dt, trial, &t);
            if (t.phi <= e.phi - 1e-4 * s * rd || s * dn <= 1e-6 * scale) { ok = 1; break; }
            s *= 0.5;
        }
        if (!ok) { *iters = it; return -1; }
        memcpy(sig, trial, sizeof trial);
        e = t;
        if (s * dn <= tol * scale) {
            memcpy(gdot, e.gdot, sizeof e.gdot);
            *iters = it;
            return 0;
        }
    }
    *iters = maxit;
    return -1;
}

int orc_newton(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
               double tauc, double dt, double tol, int maxit, double sig[6], double gdot[12], int *iters) {
    nt_flow f = {0, tauc, NULL, NULL, NULL};
    return nt_newton(p, S, M, eps_tr, &f, dt, tol, maxit, sig, gdot, iters);
}

/* Kocks-Mecking update with explicit densities and the converged shear rates (reading of the
 * paper's first and third SSD terms, Eq. SSDEvolution, with rho_F the summed density):
 *   rho^a <- rho^a + dt (k1 sqrt(rho_F) - k2 rho^a) |gdot^a|. */
void orc_km_update(const orc_params *p, double *rho, const double *gdot, double dt) {
    double rf = 0.0;
    for (int a = 0; a < 12; ++a) rf += rho[a];
    double srf = sqrt(rf);
    for (int a = 0; a < 12; ++a) rho[a] = rho[a] + dt * (p->k1 * srf - p->k2 * rho[a]) * fabs(gdot[a]);
}

static double mu_voigt(const orc_params *p) { return (p->C11 - p->C12 + 3.0 * p->C44) / 5.0; }
static double lam_voigt(const orc_params *p) { return (p->C11 + 4.0 * p->C12 - 2.0 * p->C44) / 5.0; }
static double tauc_of(const orc_params *p, const double *rho, long N3, long v) {
    double rf = 0.0;
    for (int a = 0; a < 12; ++a) rf += rho[a * N3 + v];
    return p->tau0 + p->alpha * mu_voigt(p) * p->b * sqrt(rf);
}

/* Uniaxial-stress point model of one crystal, solved by bisection on sigma33 (all other
 * stress components zero, E33 prescribed): a different algorithm from the FFT mixed-BC loop. */
int orc_point_model(const orc_params *p, const double *S, const double *M, double *sig, double *epsp,
                    double *rho, double *E, double dE33, double dt, int nsteps, double *sig33_hist) {
    for (int st = 0; st < nsteps; ++st) {
        double rf = 0.0;
        for (int a = 0; a < 12; ++a) rf += rho[a];
        double tauc = p->tau0 + p->alpha * mu_voigt(p) * p->b * sqrt(rf);
        double target = E[2] + dE33;
        nt_eval e;
        nt_flow fl = {0, tauc, NULL, NULL, NULL};
        double zero6[6] = {0, 0, 0, 0, 0, 0};
#define F33(s33, out)                                                                  \
    do {                                                                               \
        double sg[6] = {0, 0, (s33), 0, 0, 0};                                         \
        nt_evaluate(p, S, M, zero6, &fl, dt, sg, &e);                                  \
        (out) = e.r[2] + epsp[2] - target;                                             \
    } while (0)
        double lo = -1.0, hi = 1.0, flo, fhi;
        F33(lo, flo);
        F33(hi, fhi);
        for (int k = 0; k < 200 && flo > 0.0; ++k) { lo *= 2.0; F33(lo, flo); }
        for (int k = 0; k < 200 && fhi < 0.0; ++k) { hi *= 2.0; F33(hi, fhi); }
        if (flo > 0.0 || fhi < 0.0) return -1;
        for (int k = 0; k < 400 && hi - lo > 0.0; ++k) {
            double mid = 0.5 * (lo + hi), fm;
            if (mid == lo || mid == hi) break;
            F33(mid, fm);
            if (fm > 0.0) hi = mid; else lo = mid;
        }
        double s33 = 0.5 * (lo + hi);
        double sg[6] = {0, 0, s33, 0, 0, 0};
        nt_evaluate(p, S, M, zero6, &fl, dt, sg, &e);
        /* e.r = S sigma + dt eps_p_dot; total strain E = that + eps_p^t */
        for (int I = 0; I < 6; ++I) E[I] = e.r[I] + epsp[I];
        E[2] = target;
        for (int I = 0; I < 6; ++I) {
            double ep = 0.0;
            for (int a = 0; a < 12; ++a) ep += M[6 * a + I] * e.gdot[a];
            epsp[I] += dt * ep;
        }
        orc_km_update(p, rho, e.gdot, dt);
        memcpy(sig, sg, sizeof sg);
        if (sig33_hist) sig33_hist[st] = s33;
#undef F33
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Ma-Roters dislocation-density law (Sec. 2.2, Eqs. FlowRule, RhoForest, RhoParallel,
 * SSDEvolution, GNDEvolution, L0evolution, TotDislocationDensity, UpdateGND; constants of
 * Table 1). Stresses in MPa as everywhere in the oracle; the energies Q and k_B T are in J, so
 * the shear modulus enters the dimensional groups in Pa (mu_Pa = 1e6 mu).
 *
 * Readings of what the paper leaves open (each is listed with the other readings of the build):
 *  - R1 hardening frozen over an increment: rho_F, rho_P, and with them tau_pass, tau_cut and the
 *    prefactor, come from the densities at the start of the increment (as tau_c for the power law);
 *  - R2 the attempt frequency nu_D (order of the Debye frequency) and Poisson's ratio are
 *    parameters; the paper prints neither;
 *  - R3 t^a = n^a x d^a (unit line direction of the edge dislocation); |cos| and |sin| of the angle
 *    between two unit vectors are |u.v| and sqrt(1 - (u.v)^2); these are frame-invariant, so one
 *    12 x 12 table per pair type serves every grain. rho_GNDen stays 0 (zero rate, zero start), so
 *    its terms vanish;
 *  - R4 mobile density: the paper prints none; the closure of Ma and Roters (2004),
 *    rho_M = 2 k_B T / (c1 c2 c3 mu b^3) sqrt(rho_P rho_F);
 *  - R5 in the SSD law gdot stands for |gdot| (storage does not depend on the sign of slip),
 *    d_dipole takes |tau|, sigma_vm is the von Mises stress sqrt(3/2 s:s) of the voxel, gdot_vm the
 *    von Mises plastic strain rate sqrt(2/3 epsp_dot:epsp_dot); explicit Euler with the converged
 *    rates, the result clipped at 0; c6 multiplies the dipole term and c7 the climb term, the
 *    placement in the equation, whose units agree with Table 1's values (its labels are swapped);
 *  - R6 the gradient of gdot^a is taken per axis on the grid with spacing l_eff: central where both
 *    neighbours belong to the voxel's grain, one-sided where only one does, 0 where neither; "the
 *    voxel's grain" = same current grain id and same orientation (initial grain);
 *  - R7 rho_GND^a grows by dt |rho_dot_GND^a| with |rho_dot_GND|^2 = rho_dot_GNDs^2 + rho_dot_GNDet^2
 *    (the conservation law on the rates); the signed components are integrated as they are;
 *  - R8 eps_vm is the von Mises equivalent of the macroscopic strain E at the end of the increment,
 *    and l_eff is updated after the increment's GND rates are taken (l_eff starts at l0 = dx);
 *  - R9 softening on nucleation and on a PF sweep scales the GND densities (all three components)
 *    by s_soften and keeps the SSD density (Eq. UpdateGND);
 *  - R10 the Newton stopping scale adds tau_ref = min_a tau_pass^a to |sigma|.
 * ---------------------------------------------------------------------------------------- */
#define ORC_KB 1.380649e-23   /* Boltzmann constant, J/K (exact SI value) */

/* |cos| and |sin| of the angles between slip-plane normals and the sense vectors t (tables 0 and
 * 2) and the slip directions d (tables 1 and 3) of every pair of systems: tab[k*144 + 12 a + b]. */
void orc_mr_tables(double tab[576]) {
    double d[12][3], nr[12][3], t[12][3];
    orc_slip_systems(d, nr);
    for (int a = 0; a < 12; ++a) {
        t[a][0] = nr[a][1] * d[a][2] - nr[a][2] * d[a][1];
        t[a][1] = nr[a][2] * d[a][0] - nr[a][0] * d[a][2];
        t[a][2] = nr[a][0] * d[a][1] - nr[a][1] * d[a][0];
    }
    for (int a = 0; a < 12; ++a)
        for (int b = 0; b < 12; ++b) {
            double ct = fabs(nr[a][0] * t[b][0] + nr[a][1] * t[b][1] + nr[a][2] * t[b][2]);
            double cd = fabs(nr[a][0] * d[b][0] + nr[a][1] * d[b][1] + nr[a][2] * d[b][2]);
            tab[0 * 144 + 12 * a + b] = ct;
            tab[1 * 144 + 12 * a + b] = cd;
            tab[2 * 144 + 12 * a + b] = sqrt(fmax(0.0, 1.0 - ct * ct));
            tab[3 * 144 + 12 * a + b] = sqrt(fmax(0.0, 1.0 - cd * cd));
        }
}

/* Eqs. RhoForest / RhoParallel with rho_GNDen = 0. */
void orc_mr_project(const double tab[576], const double ssd[12], const double gs[12], const double ge[12],
                    double rF[12], double rP[12]) {
    for (int a = 0; a < 12; ++a) {
        double f = 0.0, q = 0.0;
        for (int b = 0; b < 12; ++b) {
            f += ssd[b] * tab[12 * a + b] + fabs(gs[b] * tab[144 + 12 * a + b]) + fabs(ge[b] * tab[12 * a + b]);
            q += ssd[b] * tab[288 + 12 * a + b] + fabs(gs[b] * tab[432 + 12 * a + b]) +
                 fabs(ge[b] * tab[288 + 12 * a + b]);
        }
        rF[a] = f;
        rP[a] = q;
    }
}

/* tau_pass = c1 mu b sqrt(rho_P), tau_cut = Q_slip sqrt(rho_F) / (c2 c3 b^2) and the prefactor
 * A = gdot_0 exp(-Q_slip / k_B T), gdot_0 = 2 k_B T nu_D sqrt(rho_P) / (c1 c3 mu b^2) (Eq. FlowRule). */
void orc_mr_frozen(const orc_params *p, const double rF[12], const double rP[12], double tp[12], double tcut[12],
                   double A[12]) {
    const double kT = ORC_KB * p->T, mu = mu_voigt(p), muPa = 1e6 * mu, b = p->b;
    for (int a = 0; a < 12; ++a) {
        tp[a] = p->c1 * mu * b * sqrt(rP[a]);
        tcut[a] = 1e-6 * p->Q_slip * sqrt(rF[a]) / (p->c2 * p->c3 * b * b);
        A[a] = 2.0 * kT * p->nu_D * sqrt(rP[a]) / (p->c1 * p->c3 * muPa * b * b) * exp(-p->Q_slip / kT);
    }
}

/* Reading R4. */
double orc_mr_rho_m(const orc_params *p, double rF, double rP) {
    const double kT = ORC_KB * p->T, muPa = 1e6 * mu_voigt(p), b = p->b;
    return 2.0 * kT / (p->c1 * p->c2 * p->c3 * muPa * b * b * b) * sqrt(rP * rF);
}

/* Eq. FlowRule: gdot = A sinh((|tau| - tp) / tcut) sign(tau) above the passing stress, else 0.
 * Also d gdot / d tau and the convex potential psi(tau) = A tcut (cosh(.) - 1) whose derivative
 * is gdot. */
double orc_mr_gdot(double tau, double tp, double tcut, double A, double *dg, double *psi) {
    const double at = fabs(tau);
    if (!(at > tp)) { *dg = 0.0; *psi = 0.0; return 0.0; }
    const double x = (at - tp) / tcut;
    *dg = A * cosh(x) / tcut;
    *psi = A * tcut * (cosh(x) - 1.0);
    return tau < 0.0 ? -A * sinh(x) : A * sinh(x);
}

/* von Mises equivalents of a Mandel stress and of a Mandel strain (rate). */
double orc_vm_stress(const double s[6]) {
    const double m = (s[0] + s[1] + s[2]) / 3.0;
    const double ss = (s[0] - m) * (s[0] - m) + (s[1] - m) * (s[1] - m) + (s[2] - m) * (s[2] - m) +
                      s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
    return sqrt(1.5 * ss);
}
double orc_vm_strain(const double e[6]) {
    const double m = (e[0] + e[1] + e[2]) / 3.0;
    const double ee = (e[0] - m) * (e[0] - m) + (e[1] - m) * (e[1] - m) + (e[2] - m) * (e[2] - m) +
                      e[3] * e[3] + e[4] * e[4] + e[5] * e[5];
    return sqrt(ee / 1.5);
}

/* Eq. SSDEvolution (reading R5): lock formation, dipole formation, athermal annihilation and
 * climb, per slip system, from the densities and projections at the start of the increment and
 * the converged resolved stresses and shear rates. */
void orc_mr_ssd_rate(const orc_params *p, const double ssd[12], const double rF[12], const double rP[12],
                     const double tau[12], const double gd[12], double svm, double gvm, double rate[12]) {
    const double kT = ORC_KB * p->T, mu = mu_voigt(p), b = p->b;
    const double climb = p->c7 * exp(-p->Q_bulk / kT) * (1e6 * svm) / kT * pow(gvm, p->c8);
    for (int a = 0; a < 12; ++a) {
        const double ag = fabs(gd[a]);
        double r = p->c4 * sqrt(rF[a]) * ag - p->c5 * ssd[a] * ag;
        if (ag > 0.0) {
            const double ddip = sqrt(3.0) * mu * b / (16.0 * PI * (1.0 - p->poisson) * fabs(tau[a]));
            r += p->c6 * ddip * orc_mr_rho_m(p, rF[a], rP[a]) * ag;
        }
        r -= climb * ssd[a] * ssd[a];
        rate[a] = r;
    }
}

/* Sample-frame slip directions d and sense vectors t = n x d of every grain (G x 12 x 3 each). */
void orc_mr_grain_vectors(int G, const double *quat, double *dv, double *tv) {
    double d[12][3], nr[12][3];
    orc_slip_systems(d, nr);
    for (int g = 0; g < G; ++g) {
        double R[9];
        orc_quat_to_R(quat + 4 * g, R);
        for (int a = 0; a < 12; ++a) {
            double t[3] = {nr[a][1] * d[a][2] - nr[a][2] * d[a][1], nr[a][2] * d[a][0] - nr[a][0] * d[a][2],
                           nr[a][0] * d[a][1] - nr[a][1] * d[a][0]};
            for (int i = 0; i < 3; ++i) {
                dv[36 * g + 3 * a + i] = R[3 * i] * d[a][0] + R[3 * i + 1] * d[a][1] + R[3 * i + 2] * d[a][2];
                tv[36 * g + 3 * a + i] = R[3 * i] * t[0] + R[3 * i + 1] * t[1] + R[3 * i + 2] * t[2];
            }
        }
    }
}

/* Eq. GNDEvolution with the differences of reading R6 at voxel v: rs = rho_dot_GNDs = -(grad gdot . t)/b,
 * re = rho_dot_GNDet = (grad gdot . d)/b of its 12 systems, gd the shear-rate field 12 x N^3 (only v and its
 * six face neighbours are read). */
void orc_mr_gnd_rates_voxel(int n, const int32_t *g, const int32_t *g0, const double *gd, const double *dv,
                            const double *tv, double leff, double b, long v, double rs[12], double re[12]) {
    const long N3 = (long)n * n * n;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((long)n * n));
    long np[3], nm[3];
    np[0] = ((x + 1) % n) + (long)n * (y + (long)n * z);
    nm[0] = ((x + n - 1) % n) + (long)n * (y + (long)n * z);
    np[1] = x + (long)n * (((y + 1) % n) + (long)n * z);
    nm[1] = x + (long)n * (((y + n - 1) % n) + (long)n * z);
    np[2] = x + (long)n * (y + (long)n * ((z + 1) % n));
    nm[2] = x + (long)n * (y + (long)n * ((z + n - 1) % n));
    int sp[3], sm[3];
    for (int i = 0; i < 3; ++i) {
        sp[i] = g[np[i]] == g[v] && g0[np[i]] == g0[v];
        sm[i] = g[nm[i]] == g[v] && g0[nm[i]] == g0[v];
    }
    const double *D = dv + 36 * (long)g0[v], *T = tv + 36 * (long)g0[v];
    for (int a = 0; a < 12; ++a) {
        const double *f = gd + a * N3;
        double grad[3];
        for (int i = 0; i < 3; ++i) {
            if (sp[i] && sm[i]) grad[i] = (f[np[i]] - f[nm[i]]) / (2.0 * leff);
            else if (sp[i]) grad[i] = (f[np[i]] - f[v]) / leff;
            else if (sm[i]) grad[i] = (f[v] - f[nm[i]]) / leff;
            else grad[i] = 0.0;
        }
        double gt = 0.0, gdd = 0.0;
        for (int i = 0; i < 3; ++i) { gt += grad[i] * T[3 * a + i]; gdd += grad[i] * D[3 * a + i]; }
        rs[a] = -gt / b;
        re[a] = gdd / b;
    }
}

/* The same over the whole grid: rs, re fields 12 x N^3. */
void orc_mr_gnd_rates(int n, const int32_t *g, const int32_t *g0, const double *gd, const double *dv,
                      const double *tv, double leff, double b, double *rs, double *re) {
    const long N3 = (long)n * n * n;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < N3; ++v) {
        double r1[12], r2[12];
        orc_mr_gnd_rates_voxel(n, g, g0, gd, dv, tv, leff, b, v, r1, r2);
        for (int a = 0; a < 12; ++a) { rs[a * N3 + v] = r1[a]; re[a * N3 + v] = r2[a]; }
    }
}

/* Eq. L0evolution with reading R8. */
double orc_mr_leff_next(double leff, const double E[6], double xi) { return leff * (1.0 + orc_vm_strain(E) / xi); }

static void mr_hardening(const orc_params *p, const double tab[576], const double ssd[12], const double gs[12],
                         const double ge[12], double rF[12], double rP[12], double tp[12], double tcut[12],
                         double A[12], double *tref) {
    orc_mr_project(tab, ssd, gs, ge, rF, rP);
    orc_mr_frozen(p, rF, rP, tp, tcut, A);
    double m = tp[0];
    for (int a = 1; a < 12; ++a) m = fmin(m, tp[a]);
    *tref = m;
}

/* Eq. TotDislocationDensity: k = sum_a rho_M^a + rho_SSD^a + rho_GND^a. */
static double mr_k(const orc_params *p, const double tab[576], const double ssd[12], const double gs[12],
                   const double ge[12], const double gnd[12]) {
    double rF[12], rP[12], k = 0.0;
    orc_mr_project(tab, ssd, gs, ge, rF, rP);
    for (int a = 0; a < 12; ++a) k += orc_mr_rho_m(p, rF[a], rP[a]) + ssd[a] + gnd[a];
    return k;
}

int orc_newton_mr(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                  const double tp[12], const double tcut[12], const double A[12], double tref, double dt,
                  double tol, int maxit, double sig[6], double gdot[12], int *iters) {
    nt_flow f = {1, tref, tp, tcut, A};
    return nt_newton(p, S, M, eps_tr, &f, dt, tol, maxit, sig, gdot, iters);
}

void orc_residual_mr(const orc_params *p, const double *S, const double *M, const double eps_tr[6],
                     const double tp[12], const double tcut[12], const double A[12], double dt,
                     const double sig[6], double r[6]) {
    nt_eval e;
    nt_flow f = {1, 0.0, tp, tcut, A};
    nt_evaluate(p, S, M, eps_tr, &f, dt, sig, &e);
    memcpy(r, e.r, sizeof e.r);
}

/* The uniaxial-stress point model of one crystal (as orc_point_model, bisection on sigma33) with
 * the Ma-Roters law: SSD densities only (a uniform crystal has no slip gradients, so no GND). */
int orc_point_model_mr(const orc_params *p, const double *S, const double *M, double *sig, double *epsp,
                       double *ssd, double *E, double dE33, double dt, int nsteps, double *sig33_hist) {
    double tab[576];
    orc_mr_tables(tab);
    const double zero12[12] = {0};
    for (int st = 0; st < nsteps; ++st) {
        double rF[12], rP[12], tp[12], tcut[12], A[12], tref;
        mr_hardening(p, tab, ssd, zero12, zero12, rF, rP, tp, tcut, A, &tref);
        nt_flow fl = {1, tref, tp, tcut, A};
        double target = E[2] + dE33;
        nt_eval e;
        double zero6[6] = {0, 0, 0, 0, 0, 0};
#define F33(s33, out)                                                                  \
    do {                                                                               \
        double sg[6] = {0, 0, (s33), 0, 0, 0};                                         \
        nt_evaluate(p, S, M, zero6, &fl, dt, sg, &e);                                  \
        (out) = e.r[2] + epsp[2] - target;                                             \
    } while (0)
        double lo = -1.0, hi = 1.0, flo, fhi;
        F33(lo, flo);
        F33(hi, fhi);
        for (int k = 0; k < 200 && flo > 0.0; ++k) { lo *= 2.0; F33(lo, flo); }
        for (int k = 0; k < 200 && fhi < 0.0; ++k) { hi *= 2.0; F33(hi, fhi); }
        if (flo > 0.0 || fhi < 0.0) return -1;
        for (int k = 0; k < 400 && hi - lo > 0.0; ++k) {
            double mid = 0.5 * (lo + hi), fm;
            if (mid == lo || mid == hi) break;
            F33(mid, fm);
            if (fm > 0.0) hi = mid; else lo = mid;
        }
#undef F33
        double s33 = 0.5 * (lo + hi);
        double sg[6] = {0, 0, s33, 0, 0, 0};
        nt_evaluate(p, S, M, zero6, &fl, dt, sg, &e);
        for (int I = 0; I < 6; ++I) E[I] = e.r[I] + epsp[I];
        E[2] = target;
        double ep[6], tau[12], rate[12];
        for (int I = 0; I < 6; ++I) {
            ep[I] = 0.0;
            for (int a = 0; a < 12; ++a) ep[I] += M[6 * a + I] * e.gdot[a];
            epsp[I] += dt * ep[I];
        }
        for (int a = 0; a < 12; ++a) {
            tau[a] = 0.0;
            for (int I = 0; I < 6; ++I) tau[a] += M[6 * a + I] * sg[I];
        }
        orc_mr_ssd_rate(p, ssd, rF, rP, tau, e.gdot, orc_vm_stress(sg), orc_vm_strain(ep), rate);
        for (int a = 0; a < 12; ++a) ssd[a] = fmax(0.0, ssd[a] + dt * rate[a]);
        memcpy(sig, sg, sizeof sg);
        if (sig33_hist) sig33_hist[st] = s33;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Full state.
 * ---------------------------------------------------------------------------------------- */
struct orc_state {
    orc_config cfg;
    orc_params p;
    int n, G, K;
    long N3;
    uint64_t seed;
    int next_id, have_prev;
    double E[6], dE_prev[6];
    double *C, *S, *M;
    int32_t *g0, *g, *draws, *ids, *ids2;
    double *eps, *epsp, *sig, *deps_prev, *rho, *k, *kappa, *eta, *eta2;
    /* phase-field grid: r = 1 (the mechanics grid; gpf and kpf are g and k) or 2 (refined, Sec. 2.4):
     * npf = r n points per edge, the active sets ids/eta live there, gpf = argmax id per PF point,
     * kpf = rho_tot interpolated onto the PF grid */
    int r, npf;
    long N3pf;
    int32_t *gpf;
    double *kpf;
    double *work_eps, *work_sig;
    double complex *spec;
    /* Ma-Roters law (cfg.law = 1): rho holds rho_SSD; signed GND components gs = rho_GNDs,
     * ge = rho_GNDet and the accumulated rho_GND (12 x N^3 each); sample-frame d and t per grain;
     * the projection tables; the effective GND length */
    double *gs, *ge, *gnd, *dv, *tv;
    double tab[576];
    double leff;
};

static void *xcalloc(size_t n, size_t sz) {
    void *p = calloc(n ? n : 1, sz);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}

/* ------------------------------------------------------------------------------------------
 * The 2:1 phase-field grid (Sec. 2.4). Both grids are cell-centred and periodic: mechanics cell i
 * spans [i, i+1) with its centre at i + 1/2; PF cell I spans [I/2, (I+1)/2), centre I/2 + 1/4.
 *  - orientation: a PF point takes the grain of the nearest mechanics point, its parent cell I/2;
 *  - smooth fields (here rho_tot, the driving force): linear interpolation along each axis between
 *    the two nearest mechanics centres, weights 3/4 (the parent) and 1/4 (the neighbour on the side
 *    of the PF centre), i.e. trilinear in 3D;
 *  - back to the mechanics grid (reading, the paper is silent): the grain id of a mechanics cell is the
 *    argmax of the order parameters summed over its eight PF children (ties to the smaller id).
 * ---------------------------------------------------------------------------------------- */
static long pf_parent(const orc_state *s, long w) {
    const int m = s->npf, r = s->r;
    const int X = (int)(w % m), Y = (int)((w / m) % m), Z = (int)(w / ((long)m * m));
    return X / r + (long)s->n * (Y / r + (long)s->n * (Z / r));
}

/* the two mechanics indices bracketing PF index I along one axis, and their weights */
static void interp_axis(int I, int n, int idx[2], double wt[2]) {
    const int i = I / 2;
    if (I % 2 == 0) { idx[0] = (i + n - 1) % n; idx[1] = i; wt[0] = 0.25; wt[1] = 0.75; }
    else { idx[0] = i; idx[1] = (i + 1) % n; wt[0] = 0.75; wt[1] = 0.25; }
}

/* kpf = trilinear interpolation of k (r = 2); the eight terms summed in the order (z, y, x) outer to
 * inner, each weight formed as (wz wy) wx */
static void pf_interp_k(orc_state *s) {
    if (s->r == 1) return;
    const int n = s->n, m = s->npf;
    for (int Z = 0; Z < m; ++Z)
        for (int Y = 0; Y < m; ++Y)
            for (int X = 0; X < m; ++X) {
                int iz[2], iy[2], ix[2];
                double wz[2], wy[2], wx[2];
                interp_axis(Z, n, iz, wz);
                interp_axis(Y, n, iy, wy);
                interp_axis(X, n, ix, wx);
                double acc = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int c = 0; c < 2; ++c)
                            acc += (wz[a] * wy[b]) * wx[c] * s->k[ix[c] + (long)n * (iy[b] + (long)n * iz[a])];
                s->kpf[X + (long)m * (Y + (long)m * Z)] = acc;
            }
}

/* g on the mechanics grid from the PF order parameters (r = 2): per cell, for each id present in any
 * of its eight children, the sum of that id's order parameter over the children in the order
 * c = dx + 2 dy + 4 dz; the largest sum wins, ties to the smaller id */
static void pf_restrict_ids(orc_state *s) {
    if (s->r == 1) return;
    const int n = s->n, m = s->npf, K = s->K;
    const long M3 = s->N3pf;
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                long ch[8];
                for (int c = 0; c < 8; ++c) {
                    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
                    ch[c] = (2 * x + dx) + (long)m * ((2 * y + dy) + (long)m * (2 * z + dz));
                }
                int best = -1;
                double bsum = 0.0;
                for (int c0 = 0; c0 < 8; ++c0)
                    for (int j0 = 0; j0 < K; ++j0) {
                        const int id = s->ids[j0 * M3 + ch[c0]];
                        if (id < 0) continue;
                        double sum = 0.0;
                        for (int c = 0; c < 8; ++c)
                            for (int j = 0; j < K; ++j)
                                if (s->ids[j * M3 + ch[c]] == id) sum += s->eta[j * M3 + ch[c]];
                        if (best < 0 || sum > bsum || (sum == bsum && id < best)) { best = id; bsum = sum; }
                    }
                s->g[x + (long)n * (y + (long)n * z)] = best;
            }
}

/* k at voxel v from its densities: sum of rho for the power law, Eq. TotDislocationDensity for the
 * Ma-Roters law. */
static void refresh_k_voxel(orc_state *s, long v) {
    const long N3 = s->N3;
    if (s->cfg.law == 1) {
        double ssd[12], gs[12], ge[12], gnd[12];
        for (int a = 0; a < 12; ++a) {
            ssd[a] = s->rho[a * N3 + v]; gs[a] = s->gs[a * N3 + v];
            ge[a] = s->ge[a * N3 + v]; gnd[a] = s->gnd[a * N3 + v];
        }
        s->k[v] = mr_k(&s->p, s->tab, ssd, gs, ge, gnd);
        return;
    }
    double kk = 0.0;
    for (int a = 0; a < 12; ++a) kk += s->rho[a * N3 + v];
    s->k[v] = kk;
}

/* Softening of recrystallised material (Eq. UpdateGND): the power law's single density family is
 * scaled by s_soften; with the Ma-Roters law the GND densities are, the SSD density is kept
 * (reading R9). k follows. */
static void soften_voxel(orc_state *s, long v) {
    const long N3 = s->N3;
    const double f = s->p.s_soften;
    for (int a = 0; a < 12; ++a) {
        if (s->cfg.law == 1) {
            s->gs[a * N3 + v] = f * s->gs[a * N3 + v];
            s->ge[a * N3 + v] = f * s->ge[a * N3 + v];
            s->gnd[a * N3 + v] = f * s->gnd[a * N3 + v];
        } else {
            s->rho[a * N3 + v] = f * s->rho[a * N3 + v];
        }
    }
    refresh_k_voxel(s, v);
}

orc_state *orc_create(const orc_config *cfg, const orc_params *p, const int32_t *g0, const double *quat,
                      uint64_t seed) {
    orc_state *s = (orc_state *)xcalloc(1, sizeof *s);
    s->cfg = *cfg;
    s->p = *p;
    s->n = cfg->n;
    s->G = cfg->grains;
    s->K = cfg->kmax;
    s->N3 = (long)cfg->n * cfg->n * cfg->n;
    s->seed = seed;
    s->next_id = s->G;
#ifdef _OPENMP
    if (cfg->nthreads > 0) omp_set_num_threads(cfg->nthreads);
#endif
    long N3 = s->N3;
    s->C = xcalloc(36 * (size_t)s->G, sizeof(double));
    s->S = xcalloc(36 * (size_t)s->G, sizeof(double));
    s->M = xcalloc(72 * (size_t)s->G, sizeof(double));
    orc_grain_tables(p, s->G, quat, s->C, s->S, s->M);
    s->g0 = xcalloc(N3, sizeof(int32_t));
    s->g = xcalloc(N3, sizeof(int32_t));
    s->draws = xcalloc(N3, sizeof(int32_t));
    s->r = cfg->pf_refine == 2 ? 2 : 1;
    s->npf = s->r * s->n;
    s->N3pf = (long)s->npf * s->npf * s->npf;
    s->ids = xcalloc((size_t)s->K * s->N3pf, sizeof(int32_t));
    s->ids2 = xcalloc((size_t)s->K * s->N3pf, sizeof(int32_t));
    s->eta = xcalloc((size_t)s->K * s->N3pf, sizeof(double));
    s->eta2 = xcalloc((size_t)s->K * s->N3pf, sizeof(double));
    s->eps = xcalloc(6 * N3, sizeof(double));
    s->epsp = xcalloc(6 * N3, sizeof(double));
    s->sig = xcalloc(6 * N3, sizeof(double));
    s->deps_prev = xcalloc(6 * N3, sizeof(double));
    s->rho = xcalloc(12 * N3, sizeof(double));
    s->k = xcalloc(N3, sizeof(double));
    s->kappa = xcalloc(N3, sizeof(double));
    s->work_eps = xcalloc(6 * N3, sizeof(double));
    s->work_sig = xcalloc(6 * N3, sizeof(double));
    s->spec = xcalloc(6 * N3, sizeof(double complex));
    if (cfg->law == 1) {
        s->gs = xcalloc(12 * N3, sizeof(double));
        s->ge = xcalloc(12 * N3, sizeof(double));
        s->gnd = xcalloc(12 * N3, sizeof(double));
        s->dv = xcalloc(36 * (size_t)s->G, sizeof(double));
        s->tv = xcalloc(36 * (size_t)s->G, sizeof(double));
        orc_mr_grain_vectors(s->G, quat, s->dv, s->tv);
        orc_mr_tables(s->tab);
        s->leff = p->dx;
    }
    for (long v = 0; v < N3; ++v) {
        s->g0[v] = g0[v];
        s->g[v] = g0[v];
        for (int a = 0; a < 12; ++a) s->rho[a * N3 + v] = p->rho0;
        refresh_k_voxel(s, v);
        /* initial nucleation strength: draw 0 from Weibull(q, kc) (Sec. 2.3, implementation) */
        s->kappa[v] = orc_weibull(orc_u01(seed, (uint64_t)v, 0), p->kc, p->q);
    }
    if (s->r == 1) {
        s->gpf = s->g;
        s->kpf = s->k;
    } else {
        s->gpf = xcalloc(s->N3pf, sizeof(int32_t));
        s->kpf = xcalloc(s->N3pf, sizeof(double));
    }
    /* initial order parameters: sharp, one grain per PF point; on the refined grid every point takes
     * the orientation (grain) of its nearest mechanics point, its parent cell (Sec. 2.4) */
    for (long w = 0; w < s->N3pf; ++w) {
        const long v = pf_parent(s, w);
        for (int j = 0; j < s->K; ++j) { s->ids[j * s->N3pf + w] = -1; s->eta[j * s->N3pf + w] = 0.0; }
        s->ids[w] = g0[v];
        s->eta[w] = 1.0;
        s->gpf[w] = g0[v];
    }
    pf_interp_k(s);
    return s;
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free(s->C); free(s->S); free(s->M); free(s->g0); free(s->g); free(s->draws); free(s->ids);
    free(s->ids2); free(s->eta); free(s->eta2); free(s->eps); free(s->epsp); free(s->sig);
    free(s->deps_prev); free(s->rho); free(s->k); free(s->kappa); free(s->work_eps);
    free(s->work_sig); free(s->spec);
    if (s->r != 1) { free(s->gpf); free(s->kpf); }
    free(s->gs); free(s->ge); free(s->gnd); free(s->dv); free(s->tv);
    free(s);
}

double *orc_field(orc_state *s, const char *name) {
    if (!strcmp(name, "eps")) return s->eps;
    if (!strcmp(name, "epsp")) return s->epsp;
    if (!strcmp(name, "sig")) return s->sig;
    if (!strcmp(name, "deps_prev")) return s->deps_prev;
    if (!strcmp(name, "rho")) return s->rho;
    if (!strcmp(name, "k")) return s->k;
    if (!strcmp(name, "kappa")) return s->kappa;
    if (!strcmp(name, "kpf")) return s->kpf;
    if (!strcmp(name, "eta")) return s->eta;
    if (!strcmp(name, "C")) return s->C;
    if (!strcmp(name, "S")) return s->S;
    if (!strcmp(name, "M")) return s->M;
    if (!strcmp(name, "E")) return s->E;
    if (!strcmp(name, "dE_prev")) return s->dE_prev;
    if (!strcmp(name, "gnds")) return s->gs;
    if (!strcmp(name, "gndet")) return s->ge;
    if (!strcmp(name, "gnd")) return s->gnd;
    if (!strcmp(name, "leff")) return &s->leff;
    return NULL;
}

int32_t *orc_ifield(orc_state *s, const char *name) {
    if (!strcmp(name, "g0")) return s->g0;
    if (!strcmp(name, "g")) return s->g;
    if (!strcmp(name, "draws")) return s->draws;
    if (!strcmp(name, "ids")) return s->ids;
    if (!strcmp(name, "gpf")) return s->gpf;
    return NULL;
}

int orc_next_id(orc_state *s) { return s->next_id; }
void orc_set_next_id(orc_state *s, int next_id) { s->next_id = next_id; }

/* Recompute k = rho_tot from the densities (after a caller overwrote them). */
void orc_refresh_derived(orc_state *s) {
    for (long v = 0; v < s->N3; ++v) refresh_k_voxel(s, v);
    pf_interp_k(s);
}

double orc_leff(orc_state *s) { return s->leff; }

/* Signed frequency of index k on an n-point axis; the Nyquist index n/2 is taken as +n/2. */
static int freq(int k, int n) { return k <= n / 2 ? k : k - n; }

/* Equilibrium residual of a transformed stress field (six full complex spectra, unnormalised):
 * returns sum_xi |xi . sigma_hat(xi)|^2 with xi = 2 pi k / N and writes the mean stress. */
static double spectral_residual(int n, const double complex *spec, double mean[6]) {
    const long N3 = (long)n * n * n;
    double acc = 0.0;
    for (int I = 0; I < 6; ++I) mean[I] = creal(spec[I * N3]) / (double)N3;
    for (int kz = 0; kz < n; ++kz)
        for (int ky = 0; ky < n; ++ky)
            for (int kx = 0; kx < n; ++kx) {
                long v = kx + (long)n * (ky + (long)n * kz);
                double xi[3] = {2.0 * PI * freq(kx, n) / n, 2.0 * PI * freq(ky, n) / n, 2.0 * PI * freq(kz, n) / n};
                double complex T[3][3];
                for (int I = 0; I < 6; ++I) {
                    T[MI[I]][MJ[I]] = spec[I * N3 + v] / mw(I);
                    T[MJ[I]][MI[I]] = spec[I * N3 + v] / mw(I);
                }
                for (int i = 0; i < 3; ++i) {
                    double complex dv = 0;
                    for (int j = 0; j < 3; ++j) dv += xi[j] * T[i][j];
                    acc += creal(dv) * creal(dv) + cimag(dv) * cimag(dv);
                }
            }
    return acc;
}

/* Stand-alone form for tests: sig is 6 x N^3 (Mandel), out = [mean stress (6), residual sum]. */
void orc_stress_residual(int n, const double *sig, double out[7]) {
    const long N3 = (long)n * n * n;
    double complex *spec = (double complex *)xcalloc(6 * N3, sizeof(double complex));
    for (int I = 0; I < 6; ++I) {
        for (long v = 0; v < N3; ++v) spec[I * N3 + v] = sig[I * N3 + v];
        orc_fft3d(n, spec + I * N3, -1);
    }
    out[6] = spectral_residual(n, spec, out);
    free(spec);
}

/* ------------------------------------------------------------------------------------------
 * One mechanical increment (Sec. 2.1): the basic Green-operator fixed point with a
 * strain-driven local Newton, under mixed macroscopic conditions (E33 prescribed, the other
 * mean stresses zero). Steps, in order, per iteration k:
 *   1. sigma^k(x) = local implicit update at eps^{k-1}(x)              (Eqs. HookeLaw, PlasticRate)
 *   2. sigma_hat = FFT(sigma^k)
 *   3. err_eq = sqrt(sum_xi |xi . sigma_hat|^2) / |sigma_hat(0)|, xi = 2 pi k / N;
 *      err_bc = |<sigma>_u| / |<sigma>|  (u = stress-controlled components)
 *   4. stop if both <= tol, or if k = max_iter
 *   5. E_u += (C0_uu)^-1 (0 - <sigma>_u)
 *   6. eps^k = eps^{k-1} - iFFT(Gamma0_hat : sigma_hat) + dE, with Gamma0_hat replaced by
 *      C0^-1 at frequencies that have a Nyquist component (Moulinec-Suquet treatment of even N)
 * After convergence the state is advanced with the converged shear rates (a7).
 * ---------------------------------------------------------------------------------------- */

/* ------------------------------------------------------------------------------------------
 * One mechanical increment by the augmented Lagrangian scheme the paper names for its solver
 * (Sec. 2.1: "augmented Lagrangian scheme adapted from Michel et al. 2000"; Michel, Moulinec,
 * Suquet 2001). Unknowns: a compatible strain eps (mean E), a local strain e and a stress-like
 * multiplier lam. With an isotropic reference medium C0 (shear mu_Voigt/al_scale, Voigt bulk):
 *   (i)   eps = E + Gamma0 * (C0 : e - lam)                      (compatibility, spectral)
 *   (ii)  sigma(e) + C0 : e = lam + C0 : eps                     (local, per voxel)
 *   (iii) lam = lam + C0 : (eps - e)
 * At the fixed point eps = e and lam = sigma(e) with div lam = 0: the same solution as the basic
 * scheme. Step (ii) is the implicit stress update with the compliance S + C0^-1 and the trial strain
 * C0^-1 (lam + C0 eps) - eps_p^t, so it reuses orc_newton. Stopping rule: the RMS of eps - e relative
 * to max(|E|, 1e-6) and of C0 (eps - e) relative to max(|<lam>|, tau0), and the mean stress on the
 * stress-controlled components, all below tol.
 * ---------------------------------------------------------------------------------------- */
/* Hardening frozen over the increment (explicit in the densities, reading R1): tau_c per voxel for
 * the power law (returns NULL); for the Ma-Roters law returns hf = rho_F, rho_P, tau_pass, tau_cut,
 * A (5 x 12 x N^3) and puts the Newton stopping scale tau_ref in tauc (reading R10). */
static double *frozen_hardening(orc_state *s, double *tauc) {
    const orc_params *p = &s->p;
    const long N3 = s->N3;
    if (s->cfg.law != 1) {
        for (long v = 0; v < N3; ++v) tauc[v] = tauc_of(p, s->rho, N3, v);
        return NULL;
    }
    double *hf = (double *)xcalloc(60 * (size_t)N3, sizeof(double));
    for (long v = 0; v < N3; ++v) {
        double ssd[12], gs[12], ge[12], h[5][12];
        for (int a = 0; a < 12; ++a) {
            ssd[a] = s->rho[a * N3 + v]; gs[a] = s->gs[a * N3 + v]; ge[a] = s->ge[a * N3 + v];
        }
        mr_hardening(p, s->tab, ssd, gs, ge, h[0], h[1], h[2], h[3], h[4], &tauc[v]);
        for (int q = 0; q < 5; ++q)
            for (int a = 0; a < 12; ++a) hf[(12 * q + a) * N3 + v] = h[q][a];
    }
    return hf;
}

/* The local Newton of voxel v with compliance S (the grain's, or S + C0^-1 in the augmented
 * Lagrangian scheme) and the frozen flow-rule data of either law. */
static int local_newton(const orc_state *s, const double *S, long v, const double *tauc, const double *hf,
                        const double etr[6], double dt, double sg[6], double gd[12], int *its) {
    const long N3 = s->N3;
    const int gr = s->g0[v];
    if (hf) {
        double tp[12], tcut[12], A[12];
        for (int a = 0; a < 12; ++a) {
            tp[a] = hf[(24 + a) * N3 + v]; tcut[a] = hf[(36 + a) * N3 + v]; A[a] = hf[(48 + a) * N3 + v];
        }
        return orc_newton_mr(&s->p, S, s->M + 72 * gr, etr, tp, tcut, A, tauc[v], dt, s->cfg.newton_tol,
                             s->cfg.newton_max, sg, gd, its);
    }
    return orc_newton(&s->p, S, s->M + 72 * gr, etr, tauc[v], dt, s->cfg.newton_tol, s->cfg.newton_max, sg, gd,
                      its);
}

/* a7 with the Ma-Roters law: plastic strain from the converged shear rates, then the densities
 * by explicit Euler: SSD by Eq. SSDEvolution from the projections at the start of the increment,
 * GND by Eq. GNDEvolution from the gradient of the converged shear-rate field (readings R5-R7),
 * and k by Eq. TotDislocationDensity. hf as in orc_increment. */
static void mr_state_update(orc_state *s, const double *sigk, const double *epsk, const double *hf, double dt) {
    const orc_params *p = &s->p;
    const long N3 = s->N3;
    double *gdf = (double *)xcalloc(12 * (size_t)N3, sizeof(double));
    double *tauf = (double *)xcalloc(12 * (size_t)N3, sizeof(double));
    double *svm = (double *)xcalloc(N3, sizeof(double));
    double *gvm = (double *)xcalloc(N3, sizeof(double));
    double *rs = (double *)xcalloc(12 * (size_t)N3, sizeof(double));
    double *re = (double *)xcalloc(12 * (size_t)N3, sizeof(double));
#pragma omp parallel for schedule(static)
    for (long v = 0; v < N3; ++v) {
        const double *M = s->M + 72 * s->g0[v];
        double sg[6], ep[6] = {0, 0, 0, 0, 0, 0};
        for (int I = 0; I < 6; ++I) sg[I] = sigk[I * N3 + v];
        for (int a = 0; a < 12; ++a) {
            double tau = 0.0, dg, psi;
            for (int I = 0; I < 6; ++I) tau += M[6 * a + I] * sg[I];
            const double gd = orc_mr_gdot(tau, hf[(24 + a) * N3 + v], hf[(36 + a) * N3 + v], hf[(48 + a) * N3 + v],
                                          &dg, &psi);
            gdf[a * N3 + v] = gd;
            tauf[a * N3 + v] = tau;
            for (int I = 0; I < 6; ++I) ep[I] += M[6 * a + I] * gd;
        }
        svm[v] = orc_vm_stress(sg);
        gvm[v] = orc_vm_strain(ep);
        for (int I = 0; I < 6; ++I) {
            s->epsp[I * N3 + v] += dt * ep[I];
            s->deps_prev[I * N3 + v] = epsk[I * N3 + v] - s->eps[I * N3 + v];
            s->eps[I * N3 + v] = epsk[I * N3 + v];
            s->sig[I * N3 + v] = sg[I];
        }
    }
    orc_mr_gnd_rates(s->n, s->g, s->g0, gdf, s->dv, s->tv, s->leff, p->b, rs, re);
#pragma omp parallel for schedule(static)
    for (long v = 0; v < N3; ++v) {
        double ssd[12], rF[12], rP[12], tau[12], gd[12], rate[12];
        for (int a = 0; a < 12; ++a) {
            ssd[a] = s->rho[a * N3 + v];
            rF[a] = hf[a * N3 + v];
            rP[a] = hf[(12 + a) * N3 + v];
            tau[a] = tauf[a * N3 + v];
            gd[a] = gdf[a * N3 + v];
        }
        orc_mr_ssd_rate(p, ssd, rF, rP, tau, gd, svm[v], gvm[v], rate);
        for (int a = 0; a < 12; ++a) {
            const long i = a * N3 + v;
            s->rho[i] = fmax(0.0, ssd[a] + dt * rate[a]);
            s->gs[i] += dt * rs[i];
            s->ge[i] += dt * re[i];
            s->gnd[i] += dt * sqrt(rs[i] * rs[i] + re[i] * re[i]);
        }
        refresh_k_voxel(s, v);
    }
    free(gdf); free(tauf); free(svm); free(gvm); free(rs); free(re);
}

static int orc_increment_al(orc_state *s, double dE33, double dt, orc_stats *out) {
    const orc_params *p = &s->p;
    const int n = s->n;
    const long N3 = s->N3;
    const double lamV = lam_voigt(p), muV = mu_voigt(p);
    const double K0 = lamV + 2.0 * muV / 3.0;
    const double mu0 = muV / (s->cfg.al_scale > 0 ? s->cfg.al_scale : 1.0), lam0 = K0 - 2.0 * mu0 / 3.0;
    int status = 0;
    memset(out, 0, sizeof *out);
    double C0[36], S0[36];
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) C0[6 * I + J] = (I < 3 && J < 3 ? lam0 : 0.0) + (I == J ? 2.0 * mu0 : 0.0);
    inv_gj(6, C0, S0);
    const int U[5] = {0, 1, 3, 4, 5};
    double C0uu[25], C0uu_inv[25];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) C0uu[5 * a + b] = C0[6 * U[a] + U[b]];
    inv_gj(5, C0uu, C0uu_inv);
    /* per-grain compliance of the local problem: S + C0^-1 */
    double *Sal = (double *)xcalloc(36 * (size_t)s->G, sizeof(double));
    for (int g = 0; g < s->G; ++g)
        for (int i = 0; i < 36; ++i) Sal[36 * g + i] = s->S[36 * g + i] + S0[i];
    double *tauc = (double *)xcalloc(N3, sizeof(double));
    double *hf = frozen_hardening(s, tauc);
    double *eps = s->work_eps, *sig = s->work_sig;
    double *e = (double *)xcalloc(6 * N3, sizeof(double));
    double *lam = (double *)xcalloc(6 * N3, sizeof(double));
    /* per-voxel squared gaps |eps - e|^2 and |C0 (eps - e)|^2, summed in voxel order after the
     * parallel loop so that the stopping rule does not depend on the number of threads */
    double *gap = (double *)xcalloc(2 * N3, sizeof(double));
    /* predictor (as in the basic scheme) */
    double dE[6];
    if (s->cfg.predictor && s->have_prev && s->dE_prev[2] != 0.0) {
        double r = dE33 / s->dE_prev[2];
        for (int I = 0; I < 6; ++I) dE[I] = r * s->dE_prev[I];
        dE[2] = dE33;
        for (long i = 0; i < 6 * N3; ++i) eps[i] = s->eps[i] + r * s->deps_prev[i];
    } else {
        double nu0 = lamV / (2.0 * (lamV + muV));
        double g[6] = {-nu0 * dE33, -nu0 * dE33, dE33, 0, 0, 0};
        memcpy(dE, g, sizeof g);
        for (int I = 0; I < 6; ++I)
            for (long v = 0; v < N3; ++v) eps[I * N3 + v] = s->eps[I * N3 + v] + dE[I];
    }
    /* start: e = eps, lam = sigma(eps) by the local update of the basic scheme */
    memcpy(sig, s->sig, 6 * N3 * sizeof(double));
    int newton_max = 0, newton_fail = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : newton_max) reduction(| : newton_fail)
    for (long v = 0; v < N3; ++v) {
        int gr = s->g0[v];
        double etr[6], sg[6], gd[12];
        for (int I = 0; I < 6; ++I) { etr[I] = eps[I * N3 + v] - s->epsp[I * N3 + v]; sg[I] = sig[I * N3 + v]; }
        int its = 0;
        if (local_newton(s, s->S + 36 * gr, v, tauc, hf, etr, dt, sg, gd, &its)) newton_fail |= 1;
        if (its > newton_max) newton_max = its;
        for (int I = 0; I < 6; ++I) { sig[I * N3 + v] = sg[I]; lam[I * N3 + v] = sg[I]; e[I * N3 + v] = eps[I * N3 + v]; }
    }
    int k, conv = 0;
    double err_cmp = 0, err_lam = 0, err_bc = 0, mean[6] = {0};
    for (k = 1; k <= s->cfg.max_iter && !newton_fail; ++k) {
        /* macroscopic strain on the stress-controlled components, from <lam> */
        for (int I = 0; I < 6; ++I) {
            double a = 0.0;
            for (long v = 0; v < N3; ++v) a += lam[I * N3 + v];
            mean[I] = a / (double)N3;
        }
        double dEk[6] = {0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 5; ++a) {
            double v = 0.0;
            for (int b = 0; b < 5; ++b) v += C0uu_inv[5 * a + b] * (0.0 - mean[U[b]]);
            dEk[U[a]] = v;
        }
        for (int I = 0; I < 6; ++I) dE[I] += dEk[I];
        /* (i) compatibility: eps = E + Gamma0 * (C0 e - lam) */
        for (int I = 0; I < 6; ++I) {
            for (long v = 0; v < N3; ++v) {
                double ce = 0.0;
                for (int J = 0; J < 6; ++J) ce += C0[6 * I + J] * e[J * N3 + v];
                s->spec[I * N3 + v] = ce - lam[I * N3 + v];
            }
            orc_fft3d(n, s->spec + I * N3, -1);
        }
        for (int kz = 0; kz < n; ++kz)
            for (int ky = 0; ky < n; ++ky)
                for (int kx = 0; kx < n; ++kx) {
                    long v = kx + (long)n * (ky + (long)n * kz);
                    double complex ph[6], eh[6];
                    for (int I = 0; I < 6; ++I) ph[I] = s->spec[I * N3 + v];
                    if (kx == 0 && ky == 0 && kz == 0) {
                        for (int I = 0; I < 6; ++I) eh[I] = 0;
                    } else {
                        double Gm[36];
                        int nyq = (n > 1) && (kx == n / 2 || ky == n / 2 || kz == n / 2);
                        if (nyq) memcpy(Gm, S0, sizeof Gm);
                        else {
                            double xi[3] = {freq(kx, n), freq(ky, n), freq(kz, n)};
                            orc_gamma0(xi, lam0, mu0, Gm);
                        }
                        for (int I = 0; I < 6; ++I) {
                            double complex a = 0;
                            for (int J = 0; J < 6; ++J) a += Gm[6 * I + J] * ph[J];
                            eh[I] = a;
                        }
                    }
                    for (int I = 0; I < 6; ++I) s->spec[I * N3 + v] = eh[I];
                }
        for (int I = 0; I < 6; ++I) {
            orc_fft3d(n, s->spec + I * N3, +1);
            for (long v = 0; v < N3; ++v)
                eps[I * N3 + v] = s->E[I] + dE[I] + creal(s->spec[I * N3 + v]) / (double)N3;
        }
        /* (ii) local problem and (iii) multiplier update */
        double acc_c = 0.0, acc_l = 0.0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : newton_max) reduction(| : newton_fail)
        for (long v = 0; v < N3; ++v) {
            int gr = s->g0[v];
            double tau[6], etr[6], sg[6], gd[12];
            for (int I = 0; I < 6; ++I) {
                double ce = 0.0;
                for (int J = 0; J < 6; ++J) ce += C0[6 * I + J] * eps[J * N3 + v];
                tau[I] = lam[I * N3 + v] + ce;
            }
            for (int I = 0; I < 6; ++I) {
                double st = 0.0;
                for (int J = 0; J < 6; ++J) st += S0[6 * I + J] * tau[J];
                etr[I] = st - s->epsp[I * N3 + v];
                sg[I] = sig[I * N3 + v];
            }
            int its = 0;
            if (local_newton(s, Sal + 36 * gr, v, tauc, hf, etr, dt, sg, gd, &its)) newton_fail |= 1;
            if (its > newton_max) newton_max = its;
            double ev[6], d[6];
            for (int I = 0; I < 6; ++I) {
                double st = 0.0;
                for (int J = 0; J < 6; ++J) st += S0[6 * I + J] * (tau[J] - sg[J]);
                ev[I] = st;                                  /* e = C0^-1 (tau - sigma) */
                d[I] = eps[I * N3 + v] - ev[I];
            }
            double gc = 0.0, gl = 0.0;
            for (int I = 0; I < 6; ++I) {
                double cd = 0.0;
                for (int J = 0; J < 6; ++J) cd += C0[6 * I + J] * d[J];
                lam[I * N3 + v] += cd;
                gl += cd * cd;
                gc += d[I] * d[I];
                e[I * N3 + v] = ev[I];
                sig[I * N3 + v] = sg[I];
            }
            gap[v] = gc;
            gap[N3 + v] = gl;
        }
        if (newton_fail) break;
        for (long v = 0; v < N3; ++v) {
            acc_c += gap[v];
            acc_l += gap[N3 + v];
        }
        double Enorm = 0.0, mn = 0.0, mu_n = 0.0;
        for (int I = 0; I < 6; ++I) Enorm += (s->E[I] + dE[I]) * (s->E[I] + dE[I]);
        for (int I = 0; I < 6; ++I) {
            double a = 0.0;
            for (long v = 0; v < N3; ++v) a += lam[I * N3 + v];
            mean[I] = a / (double)N3;
            mn += mean[I] * mean[I];
        }
        for (int a = 0; a < 5; ++a) mu_n += mean[U[a]] * mean[U[a]];
        const double den = fmax(sqrt(mn), p->tau0);
        err_cmp = sqrt(acc_c / (double)N3) / fmax(sqrt(Enorm), 1e-6);
        err_lam = sqrt(acc_l / (double)N3) / den;
        err_bc = sqrt(mu_n) / den;
        if (!isfinite(err_cmp) || !isfinite(err_lam)) { status = -5; break; }
        if (err_cmp <= s->cfg.tol && err_lam <= s->cfg.tol && err_bc <= s->cfg.tol) { conv = 1; break; }
    }
    if (newton_fail) status = -3;
    out->iterations = k > s->cfg.max_iter ? s->cfg.max_iter : k;
    out->newton_max_iters = newton_max;
    out->err_eq = err_lam;
    out->err_bc = err_bc;
    /* report the mean of the stress field itself */
    for (int I = 0; I < 6; ++I) {
        double a = 0.0;
        for (long v = 0; v < N3; ++v) a += sig[I * N3 + v];
        out->sig_mean[I] = a / (double)N3;
    }
    if (status == 0 && !conv) status = s->cfg.allow_unconverged ? 1 : -4;
    if (status < 0) {
        for (int I = 0; I < 6; ++I) out->E[I] = s->E[I] + dE[I];
        out->status = status;
        free(Sal); free(tauc); free(e); free(lam); free(hf); free(gap);
        return status;
    }
    /* state update with the converged stress; the stored total strain is the compatible field eps
     * of the last compatibility step (equal to the local strain e to the tolerance) */
    if (hf) {
        mr_state_update(s, sig, eps, hf, dt);
    } else {
#pragma omp parallel for schedule(static)
    for (long v = 0; v < N3; ++v) {
        int gr = s->g0[v];
        const double *M = s->M + 72 * gr;
        double gd[12], rho[12];
        for (int a = 0; a < 12; ++a) {
            double tau = 0.0;
            for (int I = 0; I < 6; ++I) tau += M[6 * a + I] * sig[I * N3 + v];
            double x = tau / tauc[v], ax = fabs(x);
            gd[a] = ax > 0.0 ? p->gdot0 * pow(ax, p->n) * (x < 0.0 ? -1.0 : 1.0) : 0.0;
        }
        for (int I = 0; I < 6; ++I) {
            double ep = 0.0;
            for (int a = 0; a < 12; ++a) ep += M[6 * a + I] * gd[a];
            s->epsp[I * N3 + v] += dt * ep;
        }
        for (int a = 0; a < 12; ++a) rho[a] = s->rho[a * N3 + v];
        orc_km_update(p, rho, gd, dt);
        double kk = 0.0;
        for (int a = 0; a < 12; ++a) { s->rho[a * N3 + v] = rho[a]; kk += rho[a]; }
        s->k[v] = kk;
        for (int I = 0; I < 6; ++I) {
            s->deps_prev[I * N3 + v] = eps[I * N3 + v] - s->eps[I * N3 + v];
            s->eps[I * N3 + v] = eps[I * N3 + v];
            s->sig[I * N3 + v] = sig[I * N3 + v];
        }
    }
    }
    for (int I = 0; I < 6; ++I) { s->E[I] += dE[I]; s->dE_prev[I] = dE[I]; }
    if (hf) s->leff = orc_mr_leff_next(s->leff, s->E, p->xi);
    s->have_prev = 1;
    memcpy(out->E, s->E, sizeof s->E);
    out->status = status;
    free(Sal); free(tauc); free(e); free(lam); free(hf); free(gap);
    return status;
}

int orc_increment(orc_state *s, double dE33, double dt, orc_stats *out) {
    if (s->cfg.scheme == 1) return orc_increment_al(s, dE33, dt, out);
    const orc_params *p = &s->p;
    const int n = s->n;
    const long N3 = s->N3;
    /* reference medium of the Green operator and of the mixed-BC correction: the Voigt average, or a softer
     * shear modulus mu_Voigt / ref_scale with the Voigt bulk modulus (the same converged solution; the scheme
     * converges while the reference is stiffer than half of every local stiffness) */
    const double lamV = lam_voigt(p), muV = mu_voigt(p);
    const double rs = s->cfg.ref_scale > 0.0 ? s->cfg.ref_scale : 1.0;
    const double mu0 = rs == 1.0 ? muV : muV / rs;
    const double lam0 = rs == 1.0 ? lamV : lamV + 2.0 * muV / 3.0 - 2.0 * mu0 / 3.0;
    int status = 0;
    memset(out, 0, sizeof *out);

    /* reference-medium compliance (for Nyquist frequencies) and the mixed-BC correction */
    double C0[36], S0[36];
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) C0[6 * I + J] = (I < 3 && J < 3 ? lam0 : 0.0) + (I == J ? 2.0 * mu0 : 0.0);
    inv_gj(6, C0, S0);
    const int U[5] = {0, 1, 3, 4, 5};
    double C0uu[25], C0uu_inv[25];
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) C0uu[5 * a + b] = C0[6 * U[a] + U[b]];
    inv_gj(5, C0uu, C0uu_inv);

    /* hardening frozen over the increment */
    double *tauc = (double *)xcalloc(N3, sizeof(double));
    double *hf = frozen_hardening(s, tauc);

    /* predictor: extrapolate the previous strain-increment field, else a uniform guess that is
     * the reference medium's response to dE33 under zero lateral stress */
    double dE[6];
    double *epsk = s->work_eps, *sigk = s->work_sig;
    if (s->cfg.predictor && s->have_prev && s->dE_prev[2] != 0.0) {
        double r = dE33 / s->dE_prev[2];
        for (int I = 0; I < 6; ++I) dE[I] = r * s->dE_prev[I];
        dE[2] = dE33;
        for (long i = 0; i < 6 * N3; ++i) epsk[i] = s->eps[i] + r * s->deps_prev[i];
    } else {
        double nu0 = lamV / (2.0 * (lamV + muV));   /* the Voigt medium's lateral response */
        double g[6] = {-nu0 * dE33, -nu0 * dE33, dE33, 0, 0, 0};
        memcpy(dE, g, sizeof g);
        for (int I = 0; I < 6; ++I)
            for (long v = 0; v < N3; ++v) epsk[I * N3 + v] = s->eps[I * N3 + v] + dE[I];
    }
    memcpy(sigk, s->sig, 6 * N3 * sizeof(double));

    int k, conv = 0, newton_max = 0, newton_fail = 0;
    double err_eq = 0, err_bc = 0, mean[6] = {0};
    for (k = 1; k <= s->cfg.max_iter; ++k) {
        /* 1. local stress update */
#pragma omp parallel for schedule(dynamic, 64) reduction(max : newton_max) reduction(| : newton_fail)
        for (long v = 0; v < N3; ++v) {
            int gr = s->g0[v];
            double etr[6], sg[6], gd[12];
            for (int I = 0; I < 6; ++I) {
                etr[I] = epsk[I * N3 + v] - s->epsp[I * N3 + v];
                sg[I] = sigk[I * N3 + v];
            }
            int its = 0;
            int rc = local_newton(s, s->S + 36 * gr, v, tauc, hf, etr, dt, sg, gd, &its);
            if (rc) newton_fail |= 1;
            if (its > newton_max) newton_max = its;
            for (int I = 0; I < 6; ++I) sigk[I * N3 + v] = sg[I];
        }
        if (newton_fail) { status = -3; break; }
        /* 2. forward transform of the six stress components */
        for (int I = 0; I < 6; ++I) {
            for (long v = 0; v < N3; ++v) s->spec[I * N3 + v] = sigk[I * N3 + v];
            orc_fft3d(n, s->spec + I * N3, -1);
        }
        /* 3. residuals */
        double acc = 0.0, mn = 0.0, mu_n = 0.0;
        acc = spectral_residual(n, s->spec, mean);
        for (int I = 0; I < 6; ++I) mn += mean[I] * mean[I];
        for (int a = 0; a < 5; ++a) mu_n += mean[U[a]] * mean[U[a]];
        double den = fmax(sqrt(mn), p->tau0);
        err_eq = sqrt(acc) / ((double)N3 * den);
        err_bc = sqrt(mu_n) / den;
        if (!isfinite(err_eq) || !isfinite(err_bc)) { status = -5; break; }
        if (err_eq <= s->cfg.tol && err_bc <= s->cfg.tol) { conv = 1; break; }
        if (k == s->cfg.max_iter) break;
        /* 5. macroscopic strain on the stress-controlled components */
        double dEk[6] = {0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 5; ++a) {
            double v = 0.0;
            for (int b = 0; b < 5; ++b) v += C0uu_inv[5 * a + b] * (0.0 - mean[U[b]]);
            dEk[U[a]] = v;
        }
        for (int I = 0; I < 6; ++I) dE[I] += dEk[I];
        /* 6. Green-operator correction */
        for (int kz = 0; kz < n; ++kz)
            for (int ky = 0; ky < n; ++ky)
                for (int kx = 0; kx < n; ++kx) {
                    long v = kx + (long)n * (ky + (long)n * kz);
                    double complex sh[6], eh[6];
                    for (int I = 0; I < 6; ++I) sh[I] = s->spec[I * N3 + v];
                    if (kx == 0 && ky == 0 && kz == 0) {
                        for (int I = 0; I < 6; ++I) eh[I] = 0;
                    } else {
                        double Gm[36];
                        int nyq = (n > 1) && (kx == n / 2 || ky == n / 2 || kz == n / 2);
                        if (nyq) memcpy(Gm, S0, sizeof Gm);
                        else {
                            double xi[3] = {freq(kx, n), freq(ky, n), freq(kz, n)};
                            orc_gamma0(xi, lam0, mu0, Gm);
                        }
                        for (int I = 0; I < 6; ++I) {
                            double complex a = 0;
                            for (int J = 0; J < 6; ++J) a += Gm[6 * I + J] * sh[J];
                            eh[I] = -a;
                        }
                    }
                    for (int I = 0; I < 6; ++I) s->spec[I * N3 + v] = eh[I];
                }
        for (int I = 0; I < 6; ++I) {
            orc_fft3d(n, s->spec + I * N3, +1);
            for (long v = 0; v < N3; ++v) epsk[I * N3 + v] += creal(s->spec[I * N3 + v]) / (double)N3 + dEk[I];
        }
    }
    out->iterations = k > s->cfg.max_iter ? s->cfg.max_iter : k;
    out->newton_max_iters = newton_max;
    out->err_eq = err_eq;
    out->err_bc = err_bc;
    memcpy(out->sig_mean, mean, sizeof mean);
    if (status == 0 && !conv) status = s->cfg.allow_unconverged ? 1 : -4;
    if (status < 0) {
        for (int I = 0; I < 6; ++I) out->E[I] = s->E[I] + dE[I];
        out->status = status;
        free(tauc);
        free(hf);
        return status;
    }
    if (hf) {
        mr_state_update(s, sigk, epsk, hf, dt);
    } else {
    /* a7: state update with the converged stress */
#pragma omp parallel for schedule(static)
    for (long v = 0; v < N3; ++v) {
        int gr = s->g0[v];
        const double *M = s->M + 72 * gr;
        double gd[12], rho[12];
        for (int a = 0; a < 12; ++a) {
            double tau = 0.0;
            for (int I = 0; I < 6; ++I) tau += M[6 * a + I] * sigk[I * N3 + v];
            double x = tau / tauc[v], ax = fabs(x);
            gd[a] = ax > 0.0 ? p->gdot0 * pow(ax, p->n) * (x < 0.0 ? -1.0 : 1.0) : 0.0;
        }
        for (int I = 0; I < 6; ++I) {
            double ep = 0.0;
            for (int a = 0; a < 12; ++a) ep += M[6 * a + I] * gd[a];
            s->epsp[I * N3 + v] += dt * ep;
        }
        for (int a = 0; a < 12; ++a) rho[a] = s->rho[a * N3 + v];
        orc_km_update(p, rho, gd, dt);
        double kk = 0.0;
        for (int a = 0; a < 12; ++a) { s->rho[a * N3 + v] = rho[a]; kk += rho[a]; }
        s->k[v] = kk;
        for (int I = 0; I < 6; ++I) {
            s->deps_prev[I * N3 + v] = epsk[I * N3 + v] - s->eps[I * N3 + v];
            s->eps[I * N3 + v] = epsk[I * N3 + v];
            s->sig[I * N3 + v] = sigk[I * N3 + v];
        }
    }
    }
    for (int I = 0; I < 6; ++I) { s->E[I] += dE[I]; s->dE_prev[I] = dE[I]; }
    if (hf) s->leff = orc_mr_leff_next(s->leff, s->E, p->xi);
    s->have_prev = 1;
    memcpy(out->E, s->E, sizeof s->E);
    out->status = status;
    free(tauc);
    free(hf);
    return status;
}


/* ------------------------------------------------------------------------------------------
 * Differentiation (the paper calibrates its constants by hand, Sec. 3): gradient of
 * L = sum_t (<sigma33>_t - target_t)^2 over T mechanical increments with respect to
 * theta = (k1, k2, tau0, n), by the discrete adjoint of the converged increments. Nucleation and
 * phase-field events are not part of this path (held fixed; none occur in its workloads).
 *
 * Increment t maps (eps_p^{t-1}, rho^{t-1}; theta) to sigma^t through the converged equilibrium
 * problem, then eps_p^t = eps_p^{t-1} + dt sum_a m^a gdot^a(sigma^t) and the KM update of rho.
 * Linearising the converged problem: d sigma = C_t d eps + p, C_t = K^-1 (the local Newton
 * Jacobian's inverse), p = -C_t d eps_p + dSigma/dtau_c d tau_c + dSigma/dn dn, with d eps in
 * V = {compatible fluctuations} + {uniform strains with E33 = 0} and <eta, C_t d eps + p> = 0 for
 * all eta in V. For a load sigma_bar on sigma^t the adjoint field eps_bar in V solves
 * <eta, C_t eps_bar + C_t sigma_bar> = 0 for all eta in V (the same kind of heterogeneous
 * problem, solved here by the same basic Green-operator iteration), and
 * sum_x sigma_bar . d sigma = sum_x (sigma_bar + eps_bar) . p.
 * ---------------------------------------------------------------------------------------- */

/* per-voxel local quantities at a converged stress: gdot, dgdot/dtau, C_t = K^-1 */
static void adj_local(const orc_params *p, const double *S, const double *M, double tauc, double dt,
                      const double sig[6], double gd[12], double gp[12], double lnx[12], double Ct[36]) {
    double K[36];
    for (int i = 0; i < 36; ++i) K[i] = S[i];
    for (int a = 0; a < 12; ++a) {
        double tau = 0.0;
        for (int I = 0; I < 6; ++I) tau += M[6 * a + I] * sig[I];
        double x = tau / tauc, ax = fabs(x);
        double pw = ax > 0.0 ? pow(ax, p->n) : 0.0;
        gd[a] = ax > 0.0 ? p->gdot0 * pw * (x < 0.0 ? -1.0 : 1.0) : 0.0;
        gp[a] = ax > 0.0 ? p->n * p->gdot0 * (pw / ax) / tauc : 0.0;   /* d gdot / d tau */
        lnx[a] = ax > 0.0 ? log(ax) : 0.0;
        for (int I = 0; I < 6; ++I)
            for (int J = 0; J < 6; ++J) K[6 * I + J] += dt * gp[a] * M[6 * a + I] * M[6 * a + J];
    }
    inv_gj(6, K, Ct);
}

static void matvec6(const double *A, const double *x, double *y) {
    for (int I = 0; I < 6; ++I) {
        double s = 0.0;
        for (int J = 0; J < 6; ++J) s += A[6 * I + J] * x[J];
        y[I] = s;
    }
}

/* Solve <eta, Ct eb + a> = 0 for all eta in V by the basic scheme (Gamma0, mixed-BC update). */
static int adj_solve(int n, double lam0, double mu0, const double *Ct, const double *a, double *eb, double tol,
                     int maxit, double complex *spec) {
    const long N3 = (long)n * n * n;
    double C0[36], S0[36];
    for (int I = 0; I < 6; ++I)
        for (int J = 0; J < 6; ++J) C0[6 * I + J] = (I < 3 && J < 3 ? lam0 : 0.0) + (I == J ? 2.0 * mu0 : 0.0);
    inv_gj(6, C0, S0);
    const int U[5] = {0, 1, 3, 4, 5};
    double C0uu[25], C0uu_inv[25];
    for (int x = 0; x < 5; ++x)
        for (int y = 0; y < 5; ++y) C0uu[5 * x + y] = C0[6 * U[x] + U[y]];
    inv_gj(5, C0uu, C0uu_inv);
    double *tau = (double *)xcalloc(6 * N3, sizeof(double));
    double scale = 0.0;
    for (long i = 0; i < 6 * N3; ++i) scale = fmax(scale, fabs(a[i]));
    if (scale == 0.0) { free(tau); return 0; }
    memset(eb, 0, 6 * N3 * sizeof(double));
    int it;
    for (it = 1; it <= maxit; ++it) {
        for (long v = 0; v < N3; ++v) {
            double e[6], y[6];
            for (int I = 0; I < 6; ++I) e[I] = eb[I * N3 + v];
            matvec6(Ct + 36 * v, e, y);
            for (int I = 0; I < 6; ++I) tau[I * N3 + v] = y[I] + a[I * N3 + v];
        }
        for (int I = 0; I < 6; ++I) {
            for (long v = 0; v < N3; ++v) spec[I * N3 + v] = tau[I * N3 + v];
            orc_fft3d(n, spec + I * N3, -1);
        }
        double mean[6];
        double acc = spectral_residual(n, spec, mean);
        double mu_n = 0.0;
        for (int x = 0; x < 5; ++x) mu_n += mean[U[x]] * mean[U[x]];
        double err = sqrt(acc) / ((double)N3 * scale) + sqrt(mu_n) / scale;
        if (err <= tol) break;
        double dEk[6] = {0, 0, 0, 0, 0, 0};
        for (int x = 0; x < 5; ++x) {
            double v = 0.0;
            for (int y = 0; y < 5; ++y) v += C0uu_inv[5 * x + y] * (0.0 - mean[U[y]]);
            dEk[U[x]] = v;
        }
        for (int kz = 0; kz < n; ++kz)
            for (int ky = 0; ky < n; ++ky)
                for (int kx = 0; kx < n; ++kx) {
                    long v = kx + (long)n * (ky + (long)n * kz);
                    double complex sh[6];
                    for (int I = 0; I < 6; ++I) sh[I] = spec[I * N3 + v];
                    double Gm[36];
                    if (kx == 0 && ky == 0 && kz == 0) {
                        for (int I = 0; I < 6; ++I) spec[I * N3 + v] = 0;
                        continue;
                    }
                    int nyq = (n > 1) && (kx == n / 2 || ky == n / 2 || kz == n / 2);
                    if (nyq) memcpy(Gm, S0, sizeof Gm);
                    else {
                        double xi[3] = {freq(kx, n), freq(ky, n), freq(kz, n)};
                        orc_gamma0(xi, lam0, mu0, Gm);
                    }
                    for (int I = 0; I < 6; ++I) {
                        double complex acc2 = 0;
                        for (int J = 0; J < 6; ++J) acc2 += Gm[6 * I + J] * sh[J];
                        spec[I * N3 + v] = -acc2;
                    }
                }
        for (int I = 0; I < 6; ++I) {
            orc_fft3d(n, spec + I * N3, +1);
            for (long v = 0; v < N3; ++v) eb[I * N3 + v] += creal(spec[I * N3 + v]) / (double)N3 + dEk[I];
        }
    }
    free(tau);
    return it > maxit ? -4 : 0;
}

int orc_loss_grad(const orc_config *cfg, const orc_params *p, const int32_t *g0, const double *quat, uint64_t seed,
                  int T, double dE33, double dt, const double *target, double *loss, double grad[4], double *sig33,
                  double adj_tol) {
    if (cfg->law != 0) return -1;   /* the adjoint covers the power law + Kocks-Mecking only */
    orc_state *s = orc_create(cfg, p, g0, quat, seed);
    const long N3 = s->N3;
    const int n = s->n;
    const double mu = mu_voigt(p), lam = lam_voigt(p);
    double *rho_tape = (double *)xcalloc((size_t)T * 12 * N3, sizeof(double));
    double *sig_tape = (double *)xcalloc((size_t)T * 6 * N3, sizeof(double));
    double *g = (double *)xcalloc((size_t)T, sizeof(double));
    int rc = 0;
    *loss = 0.0;
    for (int t = 0; t < T; ++t) {
        memcpy(rho_tape + (size_t)t * 12 * N3, s->rho, 12 * N3 * sizeof(double));
        orc_stats st;
        rc = orc_increment(s, dE33, dt, &st);
        if (rc < 0) goto done;
        memcpy(sig_tape + (size_t)t * 6 * N3, s->sig, 6 * N3 * sizeof(double));
        double r = st.sig_mean[2] - (target ? target[t] : 0.0);
        *loss += r * r;
        g[t] = 2.0 * r;
        if (sig33) sig33[t] = st.sig_mean[2];
    }
    if (grad) {
        double *lam_ep = (double *)xcalloc(6 * N3, sizeof(double));
        double *lam_rho = (double *)xcalloc(12 * N3, sizeof(double));
        double *sbar = (double *)xcalloc(6 * N3, sizeof(double));
        double *aa = (double *)xcalloc(6 * N3, sizeof(double));
        double *eb = (double *)xcalloc(6 * N3, sizeof(double));
        double *Ct = (double *)xcalloc(36 * N3, sizeof(double));
        double *taubar = (double *)xcalloc(N3, sizeof(double));
        double gk1 = 0, gk2 = 0, gt0 = 0, gn = 0;
        const double amb = p->alpha * mu * p->b;
        for (int t = T - 1; t >= 0 && rc == 0; --t) {
            const double *rho = rho_tape + (size_t)t * 12 * N3;
            const double *sg = sig_tape + (size_t)t * 6 * N3;
            /* explicit part of the state update at fixed sigma^t, and the adjoint load sigma_bar */
            for (long v = 0; v < N3; ++v) {
                const int gr = s->g0[v];
                const double *M = s->M + 72 * gr;
                double rf = 0.0;
                for (int a = 0; a < 12; ++a) rf += rho[a * N3 + v];
                const double srf = sqrt(rf), tc = p->tau0 + amb * srf;
                double sgv[6], gd[12], gp[12], lx[12];
                for (int I = 0; I < 6; ++I) sgv[I] = sg[I * N3 + v];
                adj_local(p, s->S + 36 * gr, M, tc, dt, sgv, gd, gp, lx, Ct + 36 * v);
                double le[6], lr[12], lr_new[12], sb[6] = {0, 0, 0, 0, 0, 0};
                for (int I = 0; I < 6; ++I) le[I] = lam_ep[I * N3 + v];
                for (int a = 0; a < 12; ++a) lr[a] = lam_rho[a * N3 + v];
                sb[2] += g[t] / (double)N3;                      /* d<sigma33>/d sigma */
                double tb = 0.0, sum_lr_gd = 0.0;
                for (int a = 0; a < 12; ++a) {
                    const double *m = M + 6 * a;
                    double mle = 0.0;
                    for (int I = 0; I < 6; ++I) mle += m[I] * le[I];
                    const double hr = p->k1 * srf - p->k2 * rho[a * N3 + v];
                    const double sgn = gd[a] < 0.0 ? -1.0 : 1.0, agd = fabs(gd[a]);
                    /* through gdot(sigma): eps_p and rho updates */
                    const double coef = dt * gp[a] * (mle + lr[a] * hr * sgn);
                    for (int I = 0; I < 6; ++I) sb[I] += coef * m[I];
                    /* direct tau_c dependence of gdot: d gdot / d tau_c = -n gdot / tau_c */
                    tb += dt * (mle * (-p->n * gd[a] / tc) + lr[a] * hr * (-p->n * agd / tc));
                    /* direct n dependence: d gdot / d n = gdot ln|x| */
                    gn += dt * (mle * gd[a] * lx[a] + lr[a] * hr * agd * lx[a]);
                    gk1 += lr[a] * dt * srf * agd;
                    gk2 += lr[a] * dt * (-rho[a * N3 + v]) * agd;
                    sum_lr_gd += lr[a] * dt * p->k1 * agd;
                }
                /* d rho^a_t / d rho^b_{t-1} = delta_ab (1 - dt k2 |gdot_a|) + dt k1 |gdot_a| / (2 sqrt(rho_F)) */
                for (int b = 0; b < 12; ++b)
                    lr_new[b] = lr[b] * (1.0 - dt * p->k2 * fabs(gd[b])) + sum_lr_gd / (2.0 * srf);
                for (int b = 0; b < 12; ++b) lam_rho[b * N3 + v] = lr_new[b];
                taubar[v] = tb;
                double av[6];
                matvec6(Ct + 36 * v, sb, av);
                for (int I = 0; I < 6; ++I) {
                    sbar[I * N3 + v] = sb[I];
                    aa[I * N3 + v] = av[I];
                }
            }
            /* adjoint equilibrium solve */
            if (adj_solve(n, lam, mu, Ct, aa, eb, adj_tol, 100000, s->spec) != 0) { rc = -4; break; }
            /* implicit part: p_bar = sigma_bar + eps_bar */
            for (long v = 0; v < N3; ++v) {
                const int gr = s->g0[v];
                const double *M = s->M + 72 * gr;
                const double *rho = rho_tape + (size_t)t * 12 * N3;
                double rf = 0.0;
                for (int a = 0; a < 12; ++a) rf += rho[a * N3 + v];
                const double srf = sqrt(rf), tc = p->tau0 + amb * srf;
                double sgv[6], gd[12], gp[12], lx[12], Cl[36];
                for (int I = 0; I < 6; ++I) sgv[I] = sg[I * N3 + v];
                adj_local(p, s->S + 36 * gr, M, tc, dt, sgv, gd, gp, lx, Cl);
                double pb[6], cp[6];
                for (int I = 0; I < 6; ++I) pb[I] = sbar[I * N3 + v] + eb[I * N3 + v];
                matvec6(Cl, pb, cp);
                for (int I = 0; I < 6; ++I) lam_ep[I * N3 + v] -= cp[I];   /* dp/d eps_p = -C_t */
                double tb = taubar[v];
                for (int a = 0; a < 12; ++a) {
                    double mc = 0.0;
                    for (int I = 0; I < 6; ++I) mc += M[6 * a + I] * cp[I];
                    tb += mc * dt * p->n * gd[a] / tc;                       /* dSigma/dtau_c */
                    gn += -mc * dt * gd[a] * lx[a];                          /* dSigma/dn */
                }
                gt0 += tb;                                                   /* tau_c = tau0 + ... */
                for (int b = 0; b < 12; ++b) lam_rho[b * N3 + v] += tb * amb / (2.0 * srf);
            }
        }
        grad[0] = gk1;
        grad[1] = gk2;
        grad[2] = gt0;
        grad[3] = gn;
        free(lam_ep); free(lam_rho); free(sbar); free(aa); free(eb); free(Ct); free(taubar);
    }
done:
    free(rho_tape);
    free(sig_tape);
    free(g);
    orc_destroy(s);
    return rc;
}

/* ------------------------------------------------------------------------------------------
 * a8: stochastic DRX nucleation (Sec. 2.3 and Appendix). A grain-boundary voxel (a face
 * neighbour carries another grain id) nucleates iff k(x) = rho_tot(x) > kappa(x)
 * (Eq. TotDislocationDensity). Nuclei get fresh ids in ascending voxel order; the voxel's
 * order parameters become {(new id, 1)}, its densities are softened by s_soften (Eq. UpdateGND
 * read for a single density family) and kappa is redrawn with k_c' = s_nucl k_c.
 * ---------------------------------------------------------------------------------------- */
static long nbr(int n, long v, int dir) {
    int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((long)n * n));
    switch (dir) {
        case 0: x = (x + n - 1) % n; break;
        case 1: x = (x + 1) % n; break;
        case 2: y = (y + n - 1) % n; break;
        case 3: y = (y + 1) % n; break;
        case 4: z = (z + n - 1) % n; break;
        default: z = (z + 1) % n; break;
    }
    return x + (long)n * (y + (long)n * z);
}

int orc_nucleate(orc_state *s, uint64_t step, int32_t *n_new) {
    (void)step;
    const long N3 = s->N3;
    const orc_params *p = &s->p;
    unsigned char *mark = (unsigned char *)xcalloc(N3, 1);
    for (long v = 0; v < N3; ++v) {
        int gb = 0;
        for (int d = 0; d < 6; ++d)
            if (s->g[nbr(s->n, v, d)] != s->g[v]) gb = 1;
        mark[v] = (unsigned char)(gb && s->k[v] > s->kappa[v]);
    }
    int cnt = 0;
    for (long v = 0; v < N3; ++v) {
        if (!mark[v]) continue;
        int id = s->next_id + cnt++;
        /* the nucleus fills the PF points of this cell: the cell itself, or its r^3 children (Sec. 2.4) */
        const int x = (int)(v % s->n), y = (int)((v / s->n) % s->n), z = (int)(v / ((long)s->n * s->n));
        for (int c = 0; c < s->r * s->r * s->r; ++c) {
            const int dx = c % s->r, dy = (c / s->r) % s->r, dz = c / (s->r * s->r);
            const long w = (s->r * x + dx) + (long)s->npf * ((s->r * y + dy) + (long)s->npf * (s->r * z + dz));
            for (int j = 0; j < s->K; ++j) { s->ids[j * s->N3pf + w] = -1; s->eta[j * s->N3pf + w] = 0.0; }
            s->ids[w] = id;
            s->eta[w] = 1.0;
            s->gpf[w] = id;
        }
        s->g[v] = id;
        soften_voxel(s, v);
        s->draws[v] += 1;
        s->kappa[v] = orc_weibull(orc_u01(s->seed, (uint64_t)v, (uint64_t)s->draws[v]), p->s_nucl * p->kc, p->q);
    }
    s->next_id += cnt;
    *n_new = cnt;
    free(mark);
    pf_interp_k(s);   /* the nuclei softened rho */
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * a9: phase field (Sec. 2.4), grid-nondimensional (lengths in dx, energies in omega_gb/dx,
 * time in dx^2/(M omega_gb)). One order parameter per grain id; ids < G are deformed grains,
 * ids >= G recrystallised. Quantitative Moelans coefficients (interface width l, energy 1):
 *   m = 6/l, kappa = 3l/4, gamma = 3/2  (Eq. GBEnergyDensity with the relations below it)
 *   f0 = sum_i (eta_i^4/4 - eta_i^2/2) + gamma sum_{i<j} eta_i^2 eta_j^2 + 1/4
 *   f_def = E' D/S, D = sum_def eta^2, R = sum_rex eta^2, S = D + R  (Eq. StoredEnergyDensity)
 *   deta_i = -L dt [ m (eta_i^3 - eta_i + 2 gamma eta_i (S2 - eta_i^2)) - kappa lap(eta_i)
 *                    + (def: 2E' eta_i R/S^2 | rex: -2E' eta_i D/S^2) ]       (Eq. PFGoverning)
 * with a periodic 7-point Laplacian and explicit Euler. E' = zeta mu b^2 rho_tot dx / omega_gb.
 * ---------------------------------------------------------------------------------------- */
static double pf_E_scale(const orc_state *s) {   /* E' per unit rho_tot; lengths in PF grid spacings dx / r */
    const orc_params *p = &s->p;
    return p->zeta * (mu_voigt(p) * 1e6) * p->b * p->b * (p->dx / s->r) / p->omega_gb;
}

/* New value of one order parameter from its value at x, its six neighbours, the local sums
 * and the local driving force; the order of operations is fixed (documented above). */
static double pf_update_one(const orc_params *p, int is_def, double e0, const double nb[6], double S2,
                            double D, double R, double Ep) {
    const double l = p->l_gb, m = 6.0 / l, kap = 0.75 * l, gam = 1.5;
    double lap = nb[0] + nb[1] + nb[2] + nb[3] + nb[4] + nb[5] - 6.0 * e0;
    double df0 = m * (e0 * e0 * e0 - e0 + 2.0 * gam * e0 * (S2 - e0 * e0));
    double S = D + R, ddef = 0.0;
    if (S > 1e-12) ddef = is_def ? 2.0 * Ep * e0 * R / (S * S) : -2.0 * Ep * e0 * D / (S * S);
    return e0 - p->L_dt * (df0 - kap * lap + ddef);
}

static double eta_at(const orc_state *s, const int32_t *ids, const double *eta, long v, int id) {
    for (int j = 0; j < s->K; ++j)
        if (ids[j * s->N3pf + v] == id) return eta[j * s->N3pf + v];
    return 0.0;
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

typedef struct { int id; double e; } cand_t;
static int cmp_keep(const void *a, const void *b) { /* eta descending, then id ascending */
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->e > y->e) return -1;
    if (x->e < y->e) return 1;
    return (x->id > y->id) - (x->id < y->id);
}
static int cmp_id(const void *a, const void *b) {
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    return (x->id > y->id) - (x->id < y->id);
}

static void pf_one_step(orc_state *s, int *overflow) {
    const long N3 = s->N3pf;
    const int K = s->K, G = s->G;
    const double Esc = pf_E_scale(s);
    int ovf = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : ovf)
    for (long v = 0; v < N3; ++v) {
        long nv[6];
        for (int d = 0; d < 6; ++d) nv[d] = nbr(s->npf, v, d);
        int cand[7 * 64];
        int nc = 0;
        long src[7] = {v, nv[0], nv[1], nv[2], nv[3], nv[4], nv[5]};
        for (int q = 0; q < 7; ++q)
            for (int j = 0; j < K; ++j) {
                int id = s->ids[j * N3 + src[q]];
                if (id >= 0) cand[nc++] = id;
            }
        qsort(cand, nc, sizeof(int), cmp_int);
        int nu = 0;
        for (int i = 0; i < nc; ++i)
            if (nu == 0 || cand[nu - 1] != cand[i]) cand[nu++] = cand[i];
        /* local sums in ascending id order */
        double S2 = 0.0, D = 0.0, R = 0.0;
        double e0s[7 * 64];
        for (int i = 0; i < nu; ++i) {
            double e0 = eta_at(s, s->ids, s->eta, v, cand[i]);
            e0s[i] = e0;
            S2 += e0 * e0;
            if (cand[i] < G) D += e0 * e0; else R += e0 * e0;
        }
        double Ep = Esc * s->kpf[v];
        cand_t out[7 * 64];
        int no = 0;
        double best = -1e300;
        int best_i = -1;
        for (int i = 0; i < nu; ++i) {
            double nb[6];
            for (int d = 0; d < 6; ++d) nb[d] = eta_at(s, s->ids, s->eta, nv[d], cand[i]);
            double en = pf_update_one(&s->p, cand[i] < G, e0s[i], nb, S2, D, R, Ep);
            if (en > best) { best = en; best_i = i; }
            if (en >= s->p.eta_drop) { out[no].id = cand[i]; out[no].e = en; ++no; }
        }
        if (no == 0 && best_i >= 0) { out[0].id = cand[best_i]; out[0].e = best; no = 1; }
        qsort(out, no, sizeof(cand_t), cmp_keep);
        if (no > K) { ovf += 1; no = K; }
        qsort(out, no, sizeof(cand_t), cmp_id);
        for (int j = 0; j < K; ++j) {
            s->ids2[j * N3 + v] = j < no ? out[j].id : -1;
            s->eta2[j * N3 + v] = j < no ? out[j].e : 0.0;
        }
    }
    int32_t *ti = s->ids; s->ids = s->ids2; s->ids2 = ti;
    double *te = s->eta; s->eta = s->eta2; s->eta2 = te;
    *overflow += ovf;
}

/* grain id = argmax over the order parameters, ties to the smaller id (Sec. 2.4, last paragraph) */
static void pf_argmax(orc_state *s) {
    const long N3 = s->N3pf;
    for (long v = 0; v < N3; ++v) {
        int bi = -1;
        double be = 0.0;
        for (int j = 0; j < s->K; ++j) {
            int id = s->ids[j * N3 + v];
            if (id < 0) continue;
            double e = s->eta[j * N3 + v];
            if (bi < 0 || e > be || (e == be && id < bi)) { bi = id; be = e; }
        }
        s->gpf[v] = bi;
    }
    pf_restrict_ids(s);
}

/* Discrete free energy whose gradient is the update above: bulk + forward-difference gradient
 * energy over the periodic grid + stored energy (Eqs. TotalFreeEnergy, GBEnergyDensity,
 * StoredEnergyDensity, nondimensional). */
double orc_pf_energy(orc_state *s) {
    const long N3 = s->N3pf;
    const int K = s->K, G = s->G;
    const double l = s->p.l_gb, m = 6.0 / l, kap = 0.75 * l, gam = 1.5, Esc = pf_E_scale(s);
    double F = 0.0;
    for (long v = 0; v < N3; ++v) {
        double f0 = 0.25, S2 = 0.0, D = 0.0;
        for (int j = 0; j < K; ++j) {
            int id = s->ids[j * N3 + v];
            if (id < 0) continue;
            double e = s->eta[j * N3 + v];
            f0 += e * e * e * e / 4.0 - e * e / 2.0;
            S2 += e * e;
            if (id < G) D += e * e;
            for (int i2 = j + 1; i2 < K; ++i2) {
                if (s->ids[i2 * N3 + v] < 0) continue;
                double e2 = s->eta[i2 * N3 + v];
                f0 += gam * e * e * e2 * e2;
            }
        }
        double fdef = S2 > 1e-12 ? Esc * s->kpf[v] * D / S2 : 0.0;
        double grad = 0.0;
        for (int d = 1; d < 6; d += 2) {
            long w = nbr(s->npf, v, d);
            /* union of ids at v and w */
            int u[128], nu = 0;
            for (int j = 0; j < K; ++j) {
                if (s->ids[j * N3 + v] >= 0) u[nu++] = s->ids[j * N3 + v];
                if (s->ids[j * N3 + w] >= 0) u[nu++] = s->ids[j * N3 + w];
            }
            qsort(u, nu, sizeof(int), cmp_int);
            for (int i = 0; i < nu; ++i) {
                if (i > 0 && u[i] == u[i - 1]) continue;
                double dv = eta_at(s, s->ids, s->eta, w, u[i]) - eta_at(s, s->ids, s->eta, v, u[i]);
                grad += dv * dv;
            }
        }
        F += m * f0 + 0.5 * kap * grad + fdef;
    }
    return F;
}

void orc_stats_now(orc_state *s, orc_pf_stats *out) {   /* on the PF grid */
    const long N3 = s->N3pf;
    long rex = 0;
    unsigned char *seen = (unsigned char *)xcalloc((size_t)s->next_id + 1, 1);
    int ng = 0;
    for (long v = 0; v < N3; ++v) {
        int g = s->gpf[v];
        if (g >= s->G) ++rex;
        if (g >= 0 && g <= s->next_id && !seen[g]) { seen[g] = 1; ++ng; }
    }
    free(seen);
    out->X_rex = (double)rex / (double)N3;
    out->n_grains = ng;
    out->F_tot = orc_pf_energy(s);
}

int orc_pf_step(orc_state *s, int nsteps, orc_pf_stats *out) {
    const long N3 = s->N3;
    int32_t *gprev = (int32_t *)xcalloc(N3, sizeof(int32_t));
    memcpy(gprev, s->g, N3 * sizeof(int32_t));
    int ovf = 0;
    pf_interp_k(s);
    for (int t = 0; t < nsteps; ++t) pf_one_step(s, &ovf);
    if (nsteps > 0) pf_argmax(s);   /* also g on the mechanics grid */
    /* sweep softening: a voxel whose grain changes from a deformed to a recrystallised one
     * over this call has its densities scaled by s_soften (reading of Eq. UpdateGND) */
    for (long v = 0; v < N3; ++v) {
        if (gprev[v] < s->G && s->g[v] >= s->G) soften_voxel(s, v);
    }
    free(gprev);
    pf_interp_k(s);
    if (out) {
        orc_stats_now(s, out);
        out->overflow = ovf;
    }
    return ovf > 0 ? 2 : 0;
}

/* Dense multi-order-parameter update (every id at every voxel, no active set): the same
 * equations with the sums over all ids in ascending order. Used to pin the sparse update. */
int orc_pf_step_dense(orc_state *s, int nsteps) {
    const long N3 = s->N3pf;
    pf_interp_k(s);
    const int NG = s->next_id, K = s->K, G = s->G;
    const double Esc = pf_E_scale(s);
    double *eta = (double *)xcalloc((size_t)NG * N3, sizeof(double));
    double *eta2 = (double *)xcalloc((size_t)NG * N3, sizeof(double));
    for (long v = 0; v < N3; ++v)
        for (int j = 0; j < K; ++j) {
            int id = s->ids[j * N3 + v];
            if (id >= 0) eta[(long)id * N3 + v] = s->eta[j * N3 + v];
        }
    for (int t = 0; t < nsteps; ++t) {
        for (long v = 0; v < N3; ++v) {
            double S2 = 0.0, D = 0.0, R = 0.0;
            for (int i = 0; i < NG; ++i) {
                double e = eta[(long)i * N3 + v];
                S2 += e * e;
                if (i < G) D += e * e; else R += e * e;
            }
            double Ep = Esc * s->kpf[v];
            for (int i = 0; i < NG; ++i) {
                double nb[6];
                for (int d = 0; d < 6; ++d) nb[d] = eta[(long)i * N3 + nbr(s->npf, v, d)];
                eta2[(long)i * N3 + v] = pf_update_one(&s->p, i < G, eta[(long)i * N3 + v], nb, S2, D, R, Ep);
            }
        }
        double *tt = eta; eta = eta2; eta2 = tt;
    }
    /* write back into the slot arrays: ids whose value is not exactly zero, ascending id */
    for (long v = 0; v < N3; ++v) {
        int j = 0;
        for (int i = 0; i < NG && j < K; ++i) {
            double e = eta[(long)i * N3 + v];
            if (e != 0.0) { s->ids[j * N3 + v] = i; s->eta[j * N3 + v] = e; ++j; }
        }
        for (; j < K; ++j) { s->ids[j * N3 + v] = -1; s->eta[j * N3 + v] = 0.0; }
    }
    pf_argmax(s);
    free(eta);
    free(eta2);
    return 0;
}
