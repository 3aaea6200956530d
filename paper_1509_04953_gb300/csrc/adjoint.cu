// Discrete adjoint of the converged mechanical increments (differentiation direction: gradient of a
// stress-strain misfit with respect to theta = (k1, k2, tau0, n); the paper itself calibrates these
// parameters against curves, Sec. 3).
//
// Increment t maps (eps_p^{t-1}, rho^{t-1}; theta) to the converged sigma^t, then advances eps_p and
// rho explicitly. Linearised at convergence: d sigma = C_t d eps + p with C_t = K^-1 (inverse of the
// local Newton Jacobian), p = -C_t d eps_p + dSigma/dtau_c d tau_c + dSigma/dn dn, d eps compatible
// with zero mean in the strain-controlled component and equilibrium <eta, d sigma> = 0 for all such
// eta. For a load sigma_bar on sigma^t the adjoint field eps_bar solves the same kind of problem
// with polarisation C_t sigma_bar (the Green operator is symmetric, so the same spectral iteration
// applies), and sum_x sigma_bar . d sigma = sum_x (sigma_bar + eps_bar) . p.
//
// Per voxel:  k_adj_prep   sigma_bar, C_t, a = C_t sigma_bar, the explicit parts of the state update
//             k_adj_tau    tau = C_t eps_bar + a  (the "stress" of the adjoint fixed point)
//             k_adj_finish p_bar = sigma_bar + eps_bar and the implicit sensitivities
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "local.cuh"

namespace evp {

namespace {

constexpr int kAT = 128;

// gdot, d gdot / d tau and ln|tau/tau_c| of the 12 systems at sigma.
template <typename TA>
__device__ __forceinline__ void slip_rates(const TA *__restrict__ M, const TA sg[6], TA tauc, const MatConst &mc,
                                           TA gd[12], TA gp[12], TA lx[12]) {
    const TA inv_tc = (TA)1 / tauc;
    const TA g0 = (TA)mc.gdot0, nn = (TA)mc.n;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        TA tau = (TA)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) tau += __ldg(M + 6 * a + i) * sg[i];
        const TA x = tau * inv_tc, ax = fabs(x);
        const TA p9 = pow_nm1(ax, mc);
        const TA p10 = p9 * ax;
        gd[a] = x < (TA)0 ? -g0 * p10 : g0 * p10;
        gp[a] = nn * g0 * p9 * inv_tc;
        lx[a] = ax > (TA)0 ? log(ax) : (TA)0;
    }
}

template <typename TA>
__device__ __forceinline__ void sym_matvec(const TA *__restrict__ Ct, long N3, long v, const TA x[6], TA y[6]) {
    TA c[21];
#pragma unroll
    for (int q = 0; q < 21; ++q) c[q] = Ct[q * N3 + v];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        TA s = (TA)0;
#pragma unroll
        for (int j = 0; j < 6; ++j) s += c[i >= j ? pk(i, j) : pk(j, i)] * x[j];
        y[i] = s;
    }
}

template <typename TA>
__global__ void __launch_bounds__(kAT) k_adj_prep(long N3, const int32_t *__restrict__ g0, const TA *__restrict__ Stab,
                                                 const TA *__restrict__ Mtab, const TA *__restrict__ rho_prev,
                                                 const TA *__restrict__ sig, const TA *__restrict__ lam_ep,
                                                 TA *__restrict__ lam_rho, TA *__restrict__ Ct, TA *__restrict__ sbar,
                                                 TA *__restrict__ aout, TA *__restrict__ taub, MatConst mc, double gb0,
                                                 double gb1, double gb2, double gb3, double gb4, double gb5,
                                                 double *__restrict__ part) {
    __shared__ double red[32];
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double pk1 = 0.0, pk2 = 0.0, pn = 0.0, pa2 = 0.0;
    if (v < N3) {
        const int g = g0[v];
        const TA *M = Mtab + 72 * (long)g;
        double rf = 0.0;
        TA rho[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            rho[a] = rho_prev[a * N3 + v];
            rf += (double)rho[a];
        }
        const double srf = sqrt(rf);
        const TA tc = (TA)(mc.tau0 + mc.alpha_mu_b * srf);
        TA sg[6], le[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            sg[i] = sig[i * N3 + v];
            le[i] = lam_ep[i * N3 + v];
        }
        TA gd[12], gp[12], lx[12];
        slip_rates(M, sg, tc, mc, gd, gp, lx);
        const TA dt = (TA)mc.dt, nn = (TA)mc.n;
        const double inv3 = 1.0 / (double)N3;
        TA sb[6] = {(TA)(gb0 * inv3), (TA)(gb1 * inv3), (TA)(gb2 * inv3), (TA)(gb3 * inv3), (TA)(gb4 * inv3),
                    (TA)(gb5 * inv3)};
        TA K[21];
        const TA *S = Stab + 36 * (long)g;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) K[pk(i, j)] = __ldg(S + 6 * i + j);
        TA tb = (TA)0, sum_lr = (TA)0;
        TA lr[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) lr[a] = lam_rho[a * N3 + v];
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            TA m[6], mle = (TA)0;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                m[i] = __ldg(M + 6 * a + i);
                mle += m[i] * le[i];
            }
            const TA hr = (TA)(mc.k1 * srf) - (TA)mc.k2 * rho[a];
            const TA sgn = gd[a] < (TA)0 ? (TA)-1 : (TA)1, agd = fabs(gd[a]);
            const TA coef = dt * gp[a] * (mle + lr[a] * hr * sgn);
#pragma unroll
            for (int i = 0; i < 6; ++i) sb[i] += coef * m[i];
            const TA sl = dt * gp[a];
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) K[pk(i, j)] += sl * m[i] * m[j];
            tb += dt * (mle * (-nn * gd[a] / tc) + lr[a] * hr * (-nn * agd / tc));
            pn += (double)(dt * (mle * gd[a] * lx[a] + lr[a] * hr * agd * lx[a]));
            pk1 += (double)lr[a] * mc.dt * srf * (double)agd;
            pk2 += (double)lr[a] * mc.dt * (-(double)rho[a]) * (double)agd;
            sum_lr += lr[a] * dt * (TA)mc.k1 * agd;
        }
        const TA inv2s = (TA)(0.5 / srf);
#pragma unroll
        for (int b = 0; b < 12; ++b)
            lam_rho[b * N3 + v] = lr[b] * ((TA)1 - dt * (TA)mc.k2 * fabs(gd[b])) + sum_lr * inv2s;
        taub[v] = tb;
        // C_t = K^-1 column by column, a = C_t sigma_bar
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            TA e[6] = {0, 0, 0, 0, 0, 0}, col[6];
            e[c] = (TA)1;
            ldl_solve<TA, TA>(K, e, col);
#pragma unroll
            for (int r = c; r < 6; ++r) Ct[pk(r, c) * N3 + v] = col[r];
        }
        TA av[6];
        ldl_solve<TA, TA>(K, sb, av);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            sbar[i * N3 + v] = sb[i];
            aout[i * N3 + v] = av[i];
            pa2 += (double)av[i] * (double)av[i];
        }
    }
    const double s1 = block_sum(pk1, red), s2 = block_sum(pk2, red), s3 = block_sum(pn, red), s4 = block_sum(pa2, red);
    if (threadIdx.x == 0) {
        part[4 * blockIdx.x] = s1;
        part[4 * blockIdx.x + 1] = s2;
        part[4 * blockIdx.x + 2] = s3;
        part[4 * blockIdx.x + 3] = s4;
    }
}

template <typename TA>
__global__ void __launch_bounds__(kAT) k_adj_tau(long N3, const TA *__restrict__ Ct, const TA *__restrict__ eb,
                                                const TA *__restrict__ a, TA *__restrict__ tau) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    TA e[6], y[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) e[i] = eb[i * N3 + v];
    sym_matvec(Ct, N3, v, e, y);
#pragma unroll
    for (int i = 0; i < 6; ++i) tau[i * N3 + v] = y[i] + a[i * N3 + v];
}

template <typename TA>
__global__ void __launch_bounds__(kAT) k_adj_finish(long N3, const int32_t *__restrict__ g0, const TA *__restrict__ Mtab,
                                                   const TA *__restrict__ rho_prev, const TA *__restrict__ sig,
                                                   const TA *__restrict__ Ct, const TA *__restrict__ sbar,
                                                   const TA *__restrict__ eb, const TA *__restrict__ taub,
                                                   TA *__restrict__ lam_ep, TA *__restrict__ lam_rho, MatConst mc,
                                                   double *__restrict__ part) {
    __shared__ double red[32];
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double pt0 = 0.0, pn = 0.0;
    if (v < N3) {
        const int g = g0[v];
        const TA *M = Mtab + 72 * (long)g;
        double rf = 0.0;
#pragma unroll
        for (int a = 0; a < 12; ++a) rf += (double)rho_prev[a * N3 + v];
        const double srf = sqrt(rf);
        const TA tc = (TA)(mc.tau0 + mc.alpha_mu_b * srf);
        TA sg[6], pb[6], cp[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            sg[i] = sig[i * N3 + v];
            pb[i] = sbar[i * N3 + v] + eb[i * N3 + v];
        }
        sym_matvec(Ct, N3, v, pb, cp);
#pragma unroll
        for (int i = 0; i < 6; ++i) lam_ep[i * N3 + v] -= cp[i];
        TA gd[12], gp[12], lx[12];
        slip_rates(M, sg, tc, mc, gd, gp, lx);
        const TA dt = (TA)mc.dt, nn = (TA)mc.n;
        TA tb = taub[v];
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            TA mc_ = (TA)0;
#pragma unroll
            for (int i = 0; i < 6; ++i) mc_ += __ldg(M + 6 * a + i) * cp[i];
            tb += mc_ * dt * nn * gd[a] / tc;
            pn += (double)(-mc_ * dt * gd[a] * lx[a]);
        }
        pt0 = (double)tb;
        const TA add = tb * (TA)(mc.alpha_mu_b / (2.0 * srf));
#pragma unroll
        for (int b = 0; b < 12; ++b) lam_rho[b * N3 + v] += add;
    }
    const double s1 = block_sum(pt0, red), s2 = block_sum(pn, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1;
        part[2 * blockIdx.x + 1] = s2;
    }
}

}  // namespace

int adj_blocks(long N3) { return (int)((N3 + kAT - 1) / kAT); }

template <typename TA>
cudaError_t adj_prep(long N3, const int32_t *g0, const TA *Stab, const TA *Mtab, const TA *rho_prev, const TA *sig,
                     const TA *lam_ep, TA *lam_rho, TA *Ct, TA *sbar, TA *a, TA *taub, MatConst mc, const double *gb6,
                     double *part, cudaStream_t s) {
    k_adj_prep<TA><<<adj_blocks(N3), kAT, 0, s>>>(N3, g0, Stab, Mtab, rho_prev, sig, lam_ep, lam_rho, Ct, sbar, a, taub,
                                                  mc, gb6[0], gb6[1], gb6[2], gb6[3], gb6[4], gb6[5], part);
    return cudaGetLastError();
}

template <typename TA> cudaError_t adj_tau(long N3, const TA *Ct, const TA *eb, const TA *a, TA *tau, cudaStream_t s) {
    k_adj_tau<TA><<<adj_blocks(N3), kAT, 0, s>>>(N3, Ct, eb, a, tau);
    return cudaGetLastError();
}

template <typename TA>
cudaError_t adj_finish(long N3, const int32_t *g0, const TA *Mtab, const TA *rho_prev, const TA *sig, const TA *Ct,
                       const TA *sbar, const TA *eb, const TA *taub, TA *lam_ep, TA *lam_rho, MatConst mc, double *part,
                       cudaStream_t s) {
    k_adj_finish<TA><<<adj_blocks(N3), kAT, 0, s>>>(N3, g0, Mtab, rho_prev, sig, Ct, sbar, eb, taub, lam_ep, lam_rho,
                                                    mc, part);
    return cudaGetLastError();
}

#define EVP_INST(TA)                                                                                                  \
    template cudaError_t adj_prep<TA>(long, const int32_t *, const TA *, const TA *, const TA *, const TA *,          \
                                      const TA *, TA *, TA *, TA *, TA *, TA *, MatConst, const double *, double *,   \
                                      cudaStream_t);                                                                  \
    template cudaError_t adj_tau<TA>(long, const TA *, const TA *, const TA *, TA *, cudaStream_t);                   \
    template cudaError_t adj_finish<TA>(long, const int32_t *, const TA *, const TA *, const TA *, const TA *,        \
                                        const TA *, const TA *, const TA *, TA *, TA *, MatConst, double *,           \
                                        cudaStream_t);
EVP_INST(float)
EVP_INST(double)
#undef EVP_INST

}  // namespace evp
