// Ma-Roters dislocation-density law (Sec. 2.2): the per-increment frozen hardening (Eqs. RhoForest,
// RhoParallel, FlowRule), the shear rates after convergence, the density update with the slip-rate
// gradients (Eqs. SSDEvolution, GNDEvolution, TotDislocationDensity) and the softening of Eq. UpdateGND.
//
// Readings of what the paper leaves open:
//  - hardening frozen over an increment (tau_pass, tau_cut from the densities at its start);
//  - t = n x d; |cos| and |sin| of the angle between unit vectors, one 12 x 12 table per pair type (the
//    angles do not depend on the grain's orientation); rho_GNDen stays 0, so its terms vanish;
//  - mobile density rho_M = 2 k_B T / (c1 c2 c3 mu b^3) sqrt(rho_P rho_F) (the closure of Ma and Roters 2004);
//  - SSD terms with |gdot|, d_dipole with |tau|, sigma_vm the voxel's von Mises stress, gdot_vm the von Mises
//    plastic strain rate; explicit Euler clipped at 0; c6 in the dipole term, c7 in the climb term;
//  - the gradient per axis with spacing l_eff: central where both neighbours are in the voxel's grain (same
//    current id and same orientation), one-sided where one is, zero where none is; periodic grid;
//  - rho_GND grows by dt sqrt(rdot_GNDs^2 + rdot_GNDet^2); softening scales the three GND fields.
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "local.cuh"

namespace evp {

namespace {

constexpr int kMR = 128;

template <typename T> __device__ __forceinline__ const MRScal<T> &scal(const MRConst &c) {
    if constexpr (sizeof(T) == 4) return c.f;
    else return c.d;
}
template <typename T> __device__ __forceinline__ T tabv(const MRConst &c, int k, int i) {
    if constexpr (sizeof(T) == 4) return c.tabf[k * 144 + i];
    else return c.tab[k * 144 + i];
}

template <typename T> __device__ __forceinline__ void load12(const T *__restrict__ f, long N3, long v, T x[12]) {
#pragma unroll
    for (int a = 0; a < 12; ++a) x[a] = f[a * N3 + v];
}

// Eq. TotDislocationDensity from the densities of one voxel (the projections of Eqs. RhoForest / RhoParallel
// row by row, rho_GNDen = 0).
template <typename T>
__device__ __forceinline__ double total_density(const MRConst &c, const T ssd[12], const T gs[12], const T ge[12],
                                                const T gnd[12]) {
    const T rm = scal<T>(c).rm_c;
    double k = 0.0;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        T f = (T)0, q = (T)0;
#pragma unroll
        for (int b = 0; b < 12; ++b) {
            const int i = 12 * a + b;
            f += ssd[b] * tabv<T>(c, 0, i) + fabs(gs[b]) * tabv<T>(c, 1, i) + fabs(ge[b]) * tabv<T>(c, 0, i);
            q += ssd[b] * tabv<T>(c, 2, i) + fabs(gs[b]) * tabv<T>(c, 3, i) + fabs(ge[b]) * tabv<T>(c, 2, i);
        }
        k += (double)(rm * sqrt(q * f)) + (double)ssd[a] + (double)gnd[a];
    }
    return k;
}

template <typename T>
__global__ void __launch_bounds__(kMR) k_mr_harden(long N3, const T *__restrict__ ssd, const T *__restrict__ gs,
                                                  const T *__restrict__ ge, T *__restrict__ tpi, T *__restrict__ tref,
                                                  MRConst c) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    T s[12], a1[12], a2[12];
    load12(ssd, N3, v, s);
    load12(gs, N3, v, a1);
    load12(ge, N3, v, a2);
    const MRScal<T> &k = scal<T>(c);
    T m = (T)0;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        T f = (T)0, q = (T)0;   // row a of Eqs. RhoForest / RhoParallel
#pragma unroll
        for (int b = 0; b < 12; ++b) {
            const int i = 12 * a + b;
            f += s[b] * tabv<T>(c, 0, i) + fabs(a1[b]) * tabv<T>(c, 1, i) + fabs(a2[b]) * tabv<T>(c, 0, i);
            q += s[b] * tabv<T>(c, 2, i) + fabs(a1[b]) * tabv<T>(c, 3, i) + fabs(a2[b]) * tabv<T>(c, 2, i);
        }
        const T t = k.tp_c * sqrt(q);
        tpi[2 * (a * N3 + v)] = t;
        tpi[2 * (a * N3 + v) + 1] = (T)1 / (k.tcut_c * sqrt(f));
        m = a == 0 ? t : fmin(m, t);
    }
    tref[v] = m;
}

// von Mises stress sqrt(3/2 s:s) and strain (rate) sqrt(2/3 e:e) of Mandel vectors.
template <typename T> __device__ __forceinline__ T vm_of(const T x[6], T f) {
    const T m = (x[0] + x[1] + x[2]) / (T)3;
    const T ss = (x[0] - m) * (x[0] - m) + (x[1] - m) * (x[1] - m) + (x[2] - m) * (x[2] - m) + x[3] * x[3] +
                 x[4] * x[4] + x[5] * x[5];
    return sqrt(f * ss);
}

template <typename T>
__global__ void __launch_bounds__(kMR) k_mr_rates(long N3, const T *__restrict__ sig, const T *__restrict__ tpi,
                                                 const int32_t *__restrict__ g0,
                                                 const T *__restrict__ Mtab, const T *__restrict__ epst,
                                                 T *__restrict__ epse, T *__restrict__ epsp, T *__restrict__ deps,
                                                 T *__restrict__ gd, T *__restrict__ aux, MatConst mc) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const T *M = Mtab + 72 * (long)g0[v];
    T sg[6], ep[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { sg[c] = sig[c * N3 + v]; ep[c] = (T)0; }
    T dt, g0r, nn;
    flow_consts(mc, dt, g0r, nn);
    const T ga = mr_ga<T>(mc);
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        T m[6], tau = (T)0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            m[i] = __ldg(M + 6 * a + i);
            tau += m[i] * sg[i];
        }
        T g, slope, psi;
        mr_flow(tau, tpi[2 * (a * N3 + v)], tpi[2 * (a * N3 + v) + 1], ga, g, slope, psi);
        gd[a * N3 + v] = g;
#pragma unroll
        for (int i = 0; i < 6; ++i) ep[i] += m[i] * g;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const T tr = epst[c * N3 + v];
        const T eo = epse[c * N3 + v];
        epsp[c * N3 + v] += dt * ep[c];
        deps[c * N3 + v] = tr - eo;
        epse[c * N3 + v] = tr - dt * ep[c];
    }
    aux[v] = vm_of(sg, (T)1.5);
    aux[N3 + v] = vm_of(ep, (T)2 / (T)3);
}

template <typename T>
__global__ void __launch_bounds__(kMR, sizeof(T) == 4 ? 4 : 1) k_mr_update(int n, int lg, const int32_t *__restrict__ g,
                                                  const int32_t *__restrict__ g0, const T *__restrict__ gd,
                                                  const T *__restrict__ aux, const T *__restrict__ sig,
                                                  const T *__restrict__ Mtab, const T *__restrict__ vec,
                                                  T *__restrict__ ssd, T *__restrict__ gs, T *__restrict__ ge,
                                                  T *__restrict__ gnd, MRConst c, T inv_l) {
    const long N3 = (long)n << (2 * lg);
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const int msk = n - 1;
    const int x = (int)(v & msk), y = (int)((v >> lg) & msk), z = (int)(v >> (2 * lg));
    const long row = v - x, pl = v - ((long)y << lg), vol = v - ((long)z << (2 * lg));
    const long np[3] = {row + ((x + 1) & msk), pl + ((long)((y + 1) & msk) << lg), vol + ((long)((z + 1) & msk) << (2 * lg))};
    const long nm[3] = {row + ((x - 1) & msk), pl + ((long)((y - 1) & msk) << lg), vol + ((long)((z - 1) & msk) << (2 * lg))};
    const int gv = g[v], ov = g0[v];
    bool sp[3], sm[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        sp[i] = g[np[i]] == gv && g0[np[i]] == ov;
        sm[i] = g[nm[i]] == gv && g0[nm[i]] == ov;
    }
    const MRScal<T> &k = scal<T>(c);
    const T *D = vec + 72 * (long)ov, *Tv = D + 36, *M = Mtab + 72 * (long)ov;
    T sg[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) sg[q] = sig[q * N3 + v];
    T s[12], a1[12], a2[12];
    load12(ssd, N3, v, s);
    load12(gs, N3, v, a1);
    load12(ge, N3, v, a2);
    const T svm = aux[v], gvm = aux[N3 + v];
    const T climb = gvm > (T)0 ? k.climb_c * svm * pow(gvm, k.c8) : (T)0;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        // row a of the projections of the densities at the start of the increment
        T rF = (T)0, rP = (T)0;
#pragma unroll
        for (int b = 0; b < 12; ++b) {
            const int i = 12 * a + b;
            rF += s[b] * tabv<T>(c, 0, i) + fabs(a1[b]) * tabv<T>(c, 1, i) + fabs(a2[b]) * tabv<T>(c, 0, i);
            rP += s[b] * tabv<T>(c, 2, i) + fabs(a1[b]) * tabv<T>(c, 3, i) + fabs(a2[b]) * tabv<T>(c, 2, i);
        }
        const T *f = gd + a * N3;
        const T f0 = f[v];
        T grad[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T fp = f[np[i]], fm = f[nm[i]];
            grad[i] = sp[i] && sm[i] ? (fp - fm) * ((T)0.5 * inv_l)
                      : sp[i]        ? (fp - f0) * inv_l
                      : sm[i]        ? (f0 - fm) * inv_l
                                     : (T)0;
        }
        T gt = (T)0, gdd = (T)0, tau = (T)0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gt += grad[i] * __ldg(Tv + 3 * a + i);
            gdd += grad[i] * __ldg(D + 3 * a + i);
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) tau += __ldg(M + 6 * a + i) * sg[i];
        const T rs = -gt * k.inv_b, re = gdd * k.inv_b;
        const T ag = fabs(f0);
        T rate = k.c4 * sqrt(rF) * ag - k.c5 * s[a] * ag;
        if (ag > (T)0) rate += k.c6 * (k.dd_c / fabs(tau)) * (k.rm_c * sqrt(rP * rF)) * ag;
        rate -= climb * s[a] * s[a];
        // the old densities stay in registers for the later rows' projections; the new ones go out
        ssd[a * N3 + v] = fmax((T)0, s[a] + k.dt * rate);
        gs[a * N3 + v] = a1[a] + k.dt * rs;
        ge[a * N3 + v] = a2[a] + k.dt * re;
        gnd[a * N3 + v] += k.dt * sqrt(rs * rs + re * re);
    }
}

template <typename T>
__global__ void __launch_bounds__(kMR, sizeof(T) == 4 ? 4 : 1) k_mr_soften(long N3, int mode, const int32_t *__restrict__ gprev,
                                                  const int32_t *__restrict__ g, int lo, const T *__restrict__ ssd,
                                                  T *__restrict__ gs, T *__restrict__ ge, T *__restrict__ gnd,
                                                  double *__restrict__ kf, MRConst c) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const bool sel = mode == 1 ? g[v] >= lo : mode == 2 ? (gprev[v] < lo && g[v] >= lo) : false;
    if (mode != 0 && !sel) return;
    T s[12], a1[12], a2[12], gn[12];
    load12(ssd, N3, v, s);
    load12(gs, N3, v, a1);
    load12(ge, N3, v, a2);
    load12(gnd, N3, v, gn);
    if (sel) {
        const T f = scal<T>(c).soften;
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            a1[a] = f * a1[a];
            a2[a] = f * a2[a];
            gn[a] = f * gn[a];
            gs[a * N3 + v] = a1[a];
            ge[a * N3 + v] = a2[a];
            gnd[a * N3 + v] = gn[a];
        }
    }
    kf[v] = total_density(c, s, a1, a2, gn);
}

inline int blocks_of(long N3) { return (int)((N3 + kMR - 1) / kMR); }

}  // namespace

template <typename T>
cudaError_t mr_harden(long N3, const T *ssd, const T *gs, const T *ge, T *tpi, T *tref, const MRConst &c,
                      cudaStream_t s) {
    k_mr_harden<T><<<blocks_of(N3), kMR, 0, s>>>(N3, ssd, gs, ge, tpi, tref, c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mr_rates(long N3, const T *sig, const T *tpi, const int32_t *g0, const T *Mtab, const T *epst,
                     T *epse, T *epsp, T *deps, T *gd, T *aux, MatConst mc, cudaStream_t s) {
    k_mr_rates<T><<<blocks_of(N3), kMR, 0, s>>>(N3, sig, tpi, g0, Mtab, epst, epse, epsp, deps, gd, aux, mc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mr_update(int n, const int32_t *g, const int32_t *g0, const T *gd, const T *aux, const T *sig,
                      const T *Mtab, const T *vec, T *ssd, T *gs, T *ge, T *gnd, double *k, const MRConst &c,
                      double leff, cudaStream_t s) {
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    const long N3 = (long)n * n * n;
    k_mr_update<T><<<blocks_of(N3), kMR, 0, s>>>(n, lg, g, g0, gd, aux, sig, Mtab, vec, ssd, gs, ge, gnd, c,
                                                 (T)(1.0 / leff));
    // k of the updated densities (Eq. TotDislocationDensity)
    k_mr_soften<T><<<blocks_of(N3), kMR, 0, s>>>(N3, 0, nullptr, nullptr, 0, ssd, gs, ge, gnd, k, c);
    return cudaGetLastError();
}

template <typename T>
cudaError_t mr_soften(long N3, int mode, const int32_t *gprev, const int32_t *g, int lo, const T *ssd, T *gs, T *ge,
                      T *gnd, double *k, const MRConst &c, cudaStream_t s) {
    k_mr_soften<T><<<blocks_of(N3), kMR, 0, s>>>(N3, mode, gprev, g, lo, ssd, gs, ge, gnd, k, c);
    return cudaGetLastError();
}

#define EVP_MR_INST(T)                                                                                            \
    template cudaError_t mr_harden<T>(long, const T *, const T *, const T *, T *, T *, const MRConst &,          \
                                      cudaStream_t);                                                            \
    template cudaError_t mr_rates<T>(long, const T *, const T *, const int32_t *, const T *, const T *, T *, T *, \
                                     T *, T *, T *, MatConst, cudaStream_t);                                    \
    template cudaError_t mr_update<T>(int, const int32_t *, const int32_t *, const T *, const T *, const T *,     \
                                      const T *, const T *, T *, T *, T *, T *, double *, const MRConst &, double, \
                                      cudaStream_t);                                                            \
    template cudaError_t mr_soften<T>(long, int, const int32_t *, const int32_t *, int, const T *, T *, T *, T *, \
                                      double *, const MRConst &, cudaStream_t);
EVP_MR_INST(float)
EVP_MR_INST(double)

}  // namespace evp
