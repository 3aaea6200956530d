// Microstructure initialisation and stochastic DRX nucleation (Sec. 2.3 and its Appendix;
// Eqs. NumCrt, NuclStrengthProb, TotDislocationDensity, UpdateGND).
//
// Random numbers: the SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014) applied to
// (seed, voxel, draw): h = F(seed ^ 0xD1B54A32D192ED03), h = F(h + phi*(voxel+1)),
// h = F(h + phi*(draw+1)), phi = 0x9E3779B97F4A7C15; u = ((h >> 11) + 0.5) 2^-53 in (0,1).
// The nucleation strength is kappa = kc' (-ln(1-u))^(1/q) (inverse Weibull CDF).
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace evp {

namespace {

__device__ __forceinline__ uint64_t sm64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t idx, uint64_t draw) {
    const uint64_t phi = 0x9E3779B97F4A7C15ULL;
    uint64_t h = sm64(seed ^ 0xD1B54A32D192ED03ULL);
    h = sm64(h + phi * (idx + 1));
    h = sm64(h + phi * (draw + 1));
    return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double weibull_inv(double u, double kc, double q) {
    return kc * pow(-log(1.0 - u), 1.0 / q);
}

// a1: periodic Voronoi. Exact int64 squared distances; ties to the smaller seed index.
__global__ void k_voronoi(int n, int G, const int64_t *__restrict__ seeds, int32_t *__restrict__ ids) {
    extern __shared__ int64_t sseed[];
    const bool in_smem = G <= 2048;
    if (in_smem)
        for (int i = threadIdx.x; i < 3 * G; i += blockDim.x) sseed[i] = seeds[i];
    __syncthreads();
    const int64_t *sd = in_smem ? sseed : seeds;
    const long N3 = (long)n * n * n;
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((long)n * n));
    const int64_t L = (int64_t)n << 16;
    const int64_t c0 = ((int64_t)x << 16) + 32768, c1 = ((int64_t)y << 16) + 32768, c2 = ((int64_t)z << 16) + 32768;
    int64_t best = INT64_MAX;
    int arg = 0;
    for (int g = 0; g < G; ++g) {
        int64_t d0 = c0 - sd[3 * g], d1 = c1 - sd[3 * g + 1], d2 = c2 - sd[3 * g + 2];
        d0 = d0 < 0 ? -d0 : d0;
        d1 = d1 < 0 ? -d1 : d1;
        d2 = d2 < 0 ? -d2 : d2;
        d0 %= L; d1 %= L; d2 %= L;
        d0 = min(d0, L - d0);
        d1 = min(d1, L - d1);
        d2 = min(d2, L - d2);
        const int64_t dd = d0 * d0 + d1 * d1 + d2 * d2;
        if (dd < best) { best = dd; arg = g; }
    }
    ids[v] = arg;
}

template <typename T>
__global__ void k_drx_init(long N3, const int32_t *__restrict__ g0, T *__restrict__ rho, double *__restrict__ k,
                           double *__restrict__ kappa, int32_t *__restrict__ g, int32_t *__restrict__ draws,
                           int32_t *__restrict__ ids, T *__restrict__ eta, int K, double rho0, double kc, double q,
                           uint64_t seed) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    double kk = 0.0;
    for (int a = 0; a < 12; ++a) {
        rho[a * N3 + v] = (T)rho0;
        kk += (double)(T)rho0;
    }
    k[v] = kk;
    kappa[v] = weibull_inv(uniform01(seed, (uint64_t)v, 0), kc, q);
    const int gi = g0[v];
    g[v] = gi;
    draws[v] = 0;
    if (ids != nullptr)   // active sets on the mechanics grid (the phase-field grid is set up by pf_init)
        for (int j = 0; j < K; ++j) {
            ids[j * N3 + v] = j == 0 ? gi : -1;
            eta[j * N3 + v] = j == 0 ? (T)1 : (T)0;
        }
}

template <typename T>
__global__ void k_refresh_k(long N3, const T *__restrict__ rho, double *__restrict__ k) {
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N3) return;
    double kk = 0.0;
    for (int a = 0; a < 12; ++a) kk += (double)rho[a * N3 + v];
    k[v] = kk;
}

constexpr int kNB = 256;   // voxels per block in the nucleation kernels

__device__ __forceinline__ bool is_nucleus(int n, long v, const int32_t *__restrict__ g, const double *__restrict__ k,
                                           const double *__restrict__ kappa) {
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((long)n * n));
    const long nn = (long)n * n;
    const int gi = g[v];
    const long xm = v - x + (x + n - 1) % n, xp = v - x + (x + 1) % n;
    const long ym = v + (long)(((y + n - 1) % n) - y) * n, yp = v + (long)(((y + 1) % n) - y) * n;
    const long zm = v + (long)(((z + n - 1) % n) - z) * nn, zp = v + (long)(((z + 1) % n) - z) * nn;
    const bool gb = g[xm] != gi || g[xp] != gi || g[ym] != gi || g[yp] != gi || g[zm] != gi || g[zp] != gi;
    return gb && (k[v] > kappa[v]);
}

// pass 1: per-block nucleus counts (reads the grain ids before this step's changes)
__global__ void __launch_bounds__(kNB) k_nucl_count(int n, const int32_t *__restrict__ g, const double *__restrict__ k,
                                                   const double *__restrict__ kappa, uint8_t *__restrict__ mark,
                                                   int32_t *__restrict__ blk_counts) {
    const long N3 = (long)n * n * n;
    const long v = (long)blockIdx.x * kNB + threadIdx.x;
    const int m = (v < N3) ? (int)is_nucleus(n, v, g, k, kappa) : 0;
    if (v < N3) mark[v] = (uint8_t)m;
    const int c = __syncthreads_count(m);
    if (threadIdx.x == 0) blk_counts[blockIdx.x] = c;
}

// pass 2: exclusive scan of the block counts (one block, fixed order)
__global__ void __launch_bounds__(1024) k_scan(const int32_t *__restrict__ cnt, int32_t *__restrict__ off, int nb,
                                              int32_t *__restrict__ total) {
    __shared__ int32_t part[1024];
    const int per = (nb + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int s = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) s += cnt[b0 + i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int run = threadIdx.x == 0 ? 0 : part[threadIdx.x - 1];
    for (int i = 0; i < per; ++i)
        if (b0 + i < nb) {
            off[b0 + i] = run;
            run += cnt[b0 + i];
        }
    if (threadIdx.x == 1023) *total = part[1023];
}

// pass 3: fresh ids in ascending voxel order, order parameter reset, softening, kappa redraw
template <typename T>
__global__ void __launch_bounds__(kNB) k_nucl_apply(int n, int r, int K, const uint8_t *__restrict__ mark,
                                                   const int32_t *__restrict__ off, int32_t *__restrict__ g,
                                                   double *__restrict__ k, double *__restrict__ kappa, T *__restrict__ rho,
                                                   int32_t *__restrict__ draws, int32_t *__restrict__ ids,
                                                   T *__restrict__ eta, int32_t *__restrict__ gpf, int next_id,
                                                   double s_soften, double kc_new, double q, uint64_t seed) {
    const long N3 = (long)n * n * n;
    __shared__ int wsum[kNB / 32];
    const long v = (long)blockIdx.x * kNB + threadIdx.x;
    const int m = (v < N3) ? mark[v] : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    if (!m) return;
    int rank = off[blockIdx.x] + __popc(bal & ((1u << lane) - 1u));
    for (int i = 0; i < w; ++i) rank += wsum[i];
    const int id = next_id + rank;
    // the nucleus fills every PF point of this voxel: itself, or its r^3 children on the refined grid
    const int pm = r * n;
    const long M3 = (long)pm * pm * pm;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((long)n * n));
    for (int c = 0; c < r * r * r; ++c) {
        const long pw = (r * x + c % r) + (long)pm * ((r * y + (c / r) % r) + (long)pm * (r * z + c / (r * r)));
        for (int j = 0; j < K; ++j) {
            ids[j * M3 + pw] = j == 0 ? id : -1;
            eta[j * M3 + pw] = j == 0 ? (T)1 : (T)0;
        }
        gpf[pw] = id;
    }
    g[v] = id;
    if (rho != nullptr) {   // nullptr: the caller softens (the Ma-Roters law's GND densities)
        double kk = 0.0;
        for (int a = 0; a < 12; ++a) {
            const T ra = (T)(s_soften * (double)rho[a * N3 + v]);
            rho[a * N3 + v] = ra;
            kk += (double)ra;
        }
        k[v] = kk;
    }
    const int d = draws[v] + 1;
    draws[v] = d;
    kappa[v] = weibull_inv(uniform01(seed, (uint64_t)v, (uint64_t)d), kc_new, q);
}

}  // namespace

cudaError_t voronoi(int n, int G, const int64_t *seeds, int32_t *ids, cudaStream_t s) {
    const long N3 = (long)n * n * n;
    const size_t sm = G <= 2048 ? sizeof(int64_t) * 3 * G : 0;
    k_voronoi<<<(int)((N3 + 255) / 256), 256, sm, s>>>(n, G, seeds, ids);
    return cudaGetLastError();
}

template <typename T>
cudaError_t drx_init(long N3, const int32_t *g0, T *rho, double *k, double *kappa, int32_t *g, int32_t *draws,
                     int32_t *ids, T *eta, int K, double rho0, double kc, double q, uint64_t seed, cudaStream_t s) {
    k_drx_init<T><<<(int)((N3 + 255) / 256), 256, 0, s>>>(N3, g0, rho, k, kappa, g, draws, ids, eta, K, rho0, kc, q, seed);
    return cudaGetLastError();
}

template <typename T> cudaError_t refresh_k(long N3, const T *rho, double *k, cudaStream_t s) {
    k_refresh_k<T><<<(int)((N3 + 255) / 256), 256, 0, s>>>(N3, rho, k);
    return cudaGetLastError();
}

int nucleate_blocks(long N3) { return (int)((N3 + kNB - 1) / kNB); }

template <typename T>
cudaError_t nucleate(int n, int r, int K, int32_t *g, double *k, double *kappa, T *rho, int32_t *draws,
                     int32_t *ids, T *eta, int32_t *gpf, int32_t *blk_counts, int32_t *blk_offsets,
                     int32_t *count_out, int next_id, double s_soften, double kc_new, double q, uint64_t seed,
                     cudaStream_t s) {
    const long N3 = (long)n * n * n;
    const int nb = nucleate_blocks(N3);
    // the mark bytes live right after the offsets (sized by the caller)
    uint8_t *mark = reinterpret_cast<uint8_t *>(blk_offsets + nb);
    k_nucl_count<<<nb, kNB, 0, s>>>(n, g, k, kappa, mark, blk_counts);
    k_scan<<<1, 1024, 0, s>>>(blk_counts, blk_offsets, nb, count_out);
    k_nucl_apply<T><<<nb, kNB, 0, s>>>(n, r, K, mark, blk_offsets, g, k, kappa, rho, draws, ids, eta, gpf, next_id,
                                       s_soften, kc_new, q, seed);
    return cudaGetLastError();
}

template cudaError_t drx_init<float>(long, const int32_t *, float *, double *, double *, int32_t *, int32_t *, int32_t *,
                                     float *, int, double, double, double, uint64_t, cudaStream_t);
template cudaError_t drx_init<double>(long, const int32_t *, double *, double *, double *, int32_t *, int32_t *,
                                      int32_t *, double *, int, double, double, double, uint64_t, cudaStream_t);
template cudaError_t refresh_k<float>(long, const float *, double *, cudaStream_t);
template cudaError_t refresh_k<double>(long, const double *, double *, cudaStream_t);
template cudaError_t nucleate<float>(int, int, int, int32_t *, double *, double *, float *, int32_t *, int32_t *,
                                     float *, int32_t *, int32_t *, int32_t *, int32_t *, int, double, double, double,
                                     uint64_t, cudaStream_t);
template cudaError_t nucleate<double>(int, int, int, int32_t *, double *, double *, double *, int32_t *, int32_t *,
                                      double *, int32_t *, int32_t *, int32_t *, int32_t *, int, double, double,
                                      double, uint64_t, cudaStream_t);

}  // namespace evp
