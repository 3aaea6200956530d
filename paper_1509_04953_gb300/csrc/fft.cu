// Hand-written 3D FFT passes for the Green-operator fixed point (Sec. 2.1: the spectral solve of
// the implicit stress update). Radix-2 butterflies in shared memory; one HBM round trip per axis:
//   x pass : real -> half spectrum, two real rows packed as one complex row
//   y pass : complex, lines along y loaded as [kx tile][y] (coalesced along kx)
//   z pass : complex, the six stress components of a [kx tile] x z slab of one ky; the forward
//            transform, the equilibrium residual, the Green-operator contraction and the inverse
//            transform run on the slab while it sits in shared memory
//   x pass : half spectrum -> real, fused with the strain update eps += field/N^3 + dE
// Spectra are [field][z|kz][ky][kx] with kx = 0..N/2 (row length N/2+1).
#include <cmath>
#include <cstdio>

#include "common.cuh"
#include "kernels.h"

namespace evp {

namespace {

constexpr int kThreads = 256;
constexpr int kRowPairs = 8;  // row pairs per CTA in the x passes

// In-place radix-2 decimation-in-time on nlines lines of length N (input bit-reversed, output
// natural order). Line l, element j lives at buf[l*ls + j]. tw[k] = exp(-2 pi i k/N), k < N/2.
template <typename C>
__device__ void fft_dit(C *buf, int N, int logN, int nlines, int ls, const C *tw, bool inverse) {
    const int half = N >> 1;
    const int nb = nlines * half;
    for (int s = 0; s < logN; ++s) {
        const int h = 1 << s;
        const int tws = half >> s;
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const int l = t >> (logN - 1), j = t & (half - 1);
            const int pos = j & (h - 1), grp = j >> s;
            const int i0 = l * ls + grp * 2 * h + pos, i1 = i0 + h;
            C w = tw[pos * tws];
            if (inverse) w.y = -w.y;
            const C a = buf[i0], b = cmul(buf[i1], w);
            buf[i0] = cadd(a, b);
            buf[i1] = csub(a, b);
        }
        __syncthreads();
    }
}

// Radix-2 decimation-in-frequency (input natural, output bit-reversed).
template <typename C>
__device__ void fft_dif(C *buf, int N, int logN, int nlines, int ls, const C *tw, bool inverse) {
    const int half = N >> 1;
    const int nb = nlines * half;
    for (int s = logN - 1; s >= 0; --s) {
        const int h = 1 << s;
        const int tws = half >> s;
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            const int l = t >> (logN - 1), j = t & (half - 1);
            const int pos = j & (h - 1), grp = j >> s;
            const int i0 = l * ls + grp * 2 * h + pos, i1 = i0 + h;
            C w = tw[pos * tws];
            if (inverse) w.y = -w.y;
            const C a = buf[i0], b = buf[i1];
            buf[i0] = cadd(a, b);
            buf[i1] = cmul(csub(a, b), w);
        }
        __syncthreads();
    }
}

// Twiddles exp(-2 pi i k/N), k < N/2, computed once per CTA into shared memory.
template <typename C>
__device__ void load_tw(C *tw_s, int N) {
    for (int k = threadIdx.x; k < (N >> 1); k += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)k / (double)N, &sn, &cs);
        tw_s[k] = cmk<C>((decltype(C::x))cs, (decltype(C::x))sn);
    }
}

// ---------------------------------------------------------------------------------------------
// x pass, real -> half spectrum. CTA = kRowPairs pairs of rows (y even, y+1) of one (field, z).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft_x_r2c(const T *__restrict__ in, typename CT<T>::type *__restrict__ out,
                                                       int N, int logN, long npairs) {
    using C = typename CT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + (N >> 1);
    const int ls = N;
    const int Hx = (N >> 1) + 1;
    load_tw(tw, N);
    const long p0 = (long)blockIdx.x * kRowPairs;
    const int np = (int)min((long)kRowPairs, npairs - p0);
    for (int t = threadIdx.x; t < np * N; t += blockDim.x) {
        const int pl = t / N, j = t - pl * N;
        const long row0 = 2 * (p0 + pl);            // global row index = (field*N + z)*N + y
        const T a = in[row0 * N + j], b = in[(row0 + 1) * N + j];
        buf[pl * ls + bitrev(j, logN)] = cmk<C>(a, b);
    }
    __syncthreads();
    fft_dit(buf, N, logN, np, ls, tw, false);
    const T h = (T)0.5;
    for (int t = threadIdx.x; t < np * Hx; t += blockDim.x) {
        const int pl = t / Hx, k = t - pl * Hx;
        const C zk = buf[pl * ls + (k & (N - 1))];
        const C zc = cconj(buf[pl * ls + ((N - k) & (N - 1))]);
        const C A = cmk<C>(h * (zk.x + zc.x), h * (zk.y + zc.y));
        const C B = cmk<C>(h * (zk.y - zc.y), -h * (zk.x - zc.x));   // (zk - zc) / 2i
        const long row0 = 2 * (p0 + pl);
        out[row0 * Hx + k] = A;
        out[(row0 + 1) * Hx + k] = B;
    }
}

// ---------------------------------------------------------------------------------------------
// x pass, half spectrum -> real (complex-to-real through the same row-pair packing).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft_x_c2r(const typename CT<T>::type *__restrict__ spec, T *__restrict__ out,
                                                       int N, int logN, long npairs, T scale, int has_add, double a0, double a1, double a2, double a3,
                                                       double a4, double a5) {
    using C = typename CT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + (N >> 1);
    const int ls = N;
    const int Hx = (N >> 1) + 1;
    load_tw(tw, N);
    const long p0 = (long)blockIdx.x * kRowPairs;
    const int np = (int)min((long)kRowPairs, npairs - p0);
    for (int t = threadIdx.x; t < np * N; t += blockDim.x) {
        const int pl = t / N, k = t - pl * N;
        const long row0 = 2 * (p0 + pl);
        C A, B;
        if (k <= (N >> 1)) {
            A = spec[row0 * Hx + k];
            B = spec[(row0 + 1) * Hx + k];
        } else {
            A = cconj(spec[row0 * Hx + (N - k)]);
            B = cconj(spec[(row0 + 1) * Hx + (N - k)]);
        }
        buf[pl * ls + bitrev(k, logN)] = cmk<C>(A.x - B.y, A.y + B.x);   // A + iB
    }
    __syncthreads();
    fft_dit(buf, N, logN, np, ls, tw, true);
    const long rows_per_field = (long)N * N;
    for (int t = threadIdx.x; t < np * N; t += blockDim.x) {
        const int pl = t / N, j = t - pl * N;
        const long row0 = 2 * (p0 + pl);
        const C z = buf[pl * ls + j];
        if (has_add) {
            const int f = (int)(row0 / rows_per_field);
            const double add = f == 0 ? a0 : f == 1 ? a1 : f == 2 ? a2 : f == 3 ? a3 : f == 4 ? a4 : a5;
            out[row0 * N + j] += z.x * scale + (T)add;
            out[(row0 + 1) * N + j] += z.y * scale + (T)add;
        } else {
            out[row0 * N + j] = z.x;
            out[(row0 + 1) * N + j] = z.y;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// y pass: CTA = (field, z, kx tile of TX columns); lines along y.
// ---------------------------------------------------------------------------------------------
template <typename T, int TX>
__global__ void __launch_bounds__(kThreads) k_fft_y(typename CT<T>::type *__restrict__ spec, int N, int logN, int inverse) {
    using C = typename CT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + (N >> 1);
    const int ls = N + 1;
    const int Hx = (N >> 1) + 1;
    const int ntiles = (Hx + TX - 1) / TX;
    const int tile = blockIdx.x % ntiles;
    const long plane = blockIdx.x / ntiles;        // field*N + z
    const int kx0 = tile * TX;
    C *base = spec + plane * (long)N * Hx;
    load_tw(tw, N);
    for (int t = threadIdx.x; t < TX * N; t += blockDim.x) {
        const int y = t / TX, xl = t - y * TX;
        const int kx = kx0 + xl;
        C v = cmk<C>(0, 0);
        if (kx < Hx) v = base[(long)y * Hx + kx];
        buf[xl * ls + bitrev(y, logN)] = v;
    }
    __syncthreads();
    fft_dit(buf, N, logN, TX, ls, tw, inverse != 0);
    for (int t = threadIdx.x; t < TX * N; t += blockDim.x) {
        const int y = t / TX, xl = t - y * TX;
        const int kx = kx0 + xl;
        if (kx < Hx) base[(long)y * Hx + kx] = buf[xl * ls + y];
    }
}

// Green operator of the isotropic reference medium applied to one spectral stress (Mandel):
// eps_kh = (n_h v_k + n_k v_h)/(2 mu0) - c n_k n_h (n.v), v = sigma.n, n = xi/|xi|,
// c = (lam0+mu0)/(mu0 (lam0+2 mu0)). At frequencies with a Nyquist component the compliance of
// the reference medium replaces it; the zero frequency is left to the macroscopic update.
// Returns -Gamma:sigma in s (in place) and accumulates |xi.sigma|^2 (xi = 2 pi k/N).
template <typename C, typename T>
__device__ __forceinline__ void gamma_point(C s[6], int kx, int ky, int kz, int N, T lam0, T mu0, T &acc, bool partner,
                                            bool apply) {
    const int fx = kx;                                   // 0..N/2
    const int fy = ky <= (N >> 1) ? ky : ky - N;
    const int fz = kz <= (N >> 1) ? kz : kz - N;
    const T r2 = (T)0.70710678118654752440;
    // tensor components
    const C t11 = s[0], t22 = s[1], t33 = s[2];
    const C t23 = cmk<C>(s[3].x * r2, s[3].y * r2), t13 = cmk<C>(s[4].x * r2, s[4].y * r2),
            t12 = cmk<C>(s[5].x * r2, s[5].y * r2);
    {   // equilibrium residual |xi.sigma_hat|^2 at this frequency and, for 0 < kx < N/2, at its
        // Hermitian partner -k (whose signed frequency differs from -xi on Nyquist ky / kz planes)
        const T w = (T)(6.283185307179586476925 / N);
        const int nparts = partner ? 2 : 1;
        for (int pt = 0; pt < nparts; ++pt) {
            const int gy = pt == 0 ? fy : ((N - ky) % N <= (N >> 1) ? (N - ky) % N : (N - ky) % N - N);
            const int gz = pt == 0 ? fz : ((N - kz) % N <= (N >> 1) ? (N - kz) % N : (N - kz) % N - N);
            const T x1 = w * (pt == 0 ? fx : -fx), x2 = w * gy, x3 = w * gz;
            const C d1 = cmk<C>(x1 * t11.x + x2 * t12.x + x3 * t13.x, x1 * t11.y + x2 * t12.y + x3 * t13.y);
            const C d2 = cmk<C>(x1 * t12.x + x2 * t22.x + x3 * t23.x, x1 * t12.y + x2 * t22.y + x3 * t23.y);
            const C d3 = cmk<C>(x1 * t13.x + x2 * t23.x + x3 * t33.x, x1 * t13.y + x2 * t23.y + x3 * t33.y);
            acc += d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y + d3.x * d3.x + d3.y * d3.y;
        }
    }
    if (!apply) return;
    if (fx == 0 && fy == 0 && fz == 0) {
        for (int i = 0; i < 6; ++i) s[i] = cmk<C>(0, 0);
        return;
    }
    const int h = N >> 1;
    if (kx == h || ky == h || kz == h) {
        // -S0:sigma, S0 = (1/2mu0)(I - lam0/(3 lam0 + 2 mu0) J)
        const T a = (T)1 / ((T)2 * mu0), b = lam0 / ((T)2 * mu0 * ((T)3 * lam0 + (T)2 * mu0));
        const C tr = cmk<C>(s[0].x + s[1].x + s[2].x, s[0].y + s[1].y + s[2].y);
        for (int i = 0; i < 3; ++i) s[i] = cmk<C>(-(a * s[i].x - b * tr.x), -(a * s[i].y - b * tr.y));
        for (int i = 3; i < 6; ++i) s[i] = cmk<C>(-a * s[i].x, -a * s[i].y);
        return;
    }
    const T inv = (T)1 / sqrt((T)(fx * fx + fy * fy + fz * fz));
    const T n1 = fx * inv, n2 = fy * inv, n3 = fz * inv;
    const C v1 = cmk<C>(t11.x * n1 + t12.x * n2 + t13.x * n3, t11.y * n1 + t12.y * n2 + t13.y * n3);
    const C v2 = cmk<C>(t12.x * n1 + t22.x * n2 + t23.x * n3, t12.y * n1 + t22.y * n2 + t23.y * n3);
    const C v3 = cmk<C>(t13.x * n1 + t23.x * n2 + t33.x * n3, t13.y * n1 + t23.y * n2 + t33.y * n3);
    const C nv = cmk<C>(n1 * v1.x + n2 * v2.x + n3 * v3.x, n1 * v1.y + n2 * v2.y + n3 * v3.y);
    const T im = (T)1 / mu0, ih = (T)0.5 / mu0;
    const T c = (lam0 + mu0) / (mu0 * (lam0 + (T)2 * mu0));
    const T sq2 = (T)1.41421356237309504880;
#define EVP_EPS_KH(nk, vk, nh, vh, diag)                                                              \
    cmk<C>(((diag) ? im * nk * vk.x : ih * (nh * vk.x + nk * vh.x)) - c * nk * nh * nv.x,             \
           ((diag) ? im * nk * vk.y : ih * (nh * vk.y + nk * vh.y)) - c * nk * nh * nv.y)
    const C e11 = EVP_EPS_KH(n1, v1, n1, v1, true);
    const C e22 = EVP_EPS_KH(n2, v2, n2, v2, true);
    const C e33 = EVP_EPS_KH(n3, v3, n3, v3, true);
    const C e23 = EVP_EPS_KH(n2, v2, n3, v3, false);
    const C e13 = EVP_EPS_KH(n1, v1, n3, v3, false);
    const C e12 = EVP_EPS_KH(n1, v1, n2, v2, false);
#undef EVP_EPS_KH
    s[0] = cmk<C>(-e11.x, -e11.y);
    s[1] = cmk<C>(-e22.x, -e22.y);
    s[2] = cmk<C>(-e33.x, -e33.y);
    s[3] = cmk<C>(-sq2 * e23.x, -sq2 * e23.y);
    s[4] = cmk<C>(-sq2 * e13.x, -sq2 * e13.y);
    s[5] = cmk<C>(-sq2 * e12.x, -sq2 * e12.y);
}

// ---------------------------------------------------------------------------------------------
// z pass: CTA = (ky, kx tile); nf fields x TX columns x N planes in shared memory.
// ---------------------------------------------------------------------------------------------
template <typename T, int TX>
__global__ void __launch_bounds__(kThreads) k_fft_z(typename CT<T>::type *__restrict__ spec, int N, int logN, int nf, int mode, T lam0, T mu0,
                                                   double *__restrict__ partials, double *__restrict__ mean6) {
    using C = typename CT<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + (N >> 1);
    __shared__ double red[32];
    const int ls = N + 1;
    const int Hx = (N >> 1) + 1;
    const int ntiles = (Hx + TX - 1) / TX;
    const int tile = blockIdx.x % ntiles;
    const int ky = blockIdx.x / ntiles;
    const int kx0 = tile * TX;
    const long plane = (long)N * Hx;            // one z plane of one field
    const long fstride = plane * N;
    load_tw(tw, N);
    for (int t = threadIdx.x; t < nf * TX * N; t += blockDim.x) {
        const int f = t / (TX * N);
        const int r = t - f * TX * N;
        const int z = r / TX, xl = r - z * TX;
        const int kx = kx0 + xl;
        C v = cmk<C>(0, 0);
        if (kx < Hx) v = spec[f * fstride + z * plane + (long)ky * Hx + kx];
        const int zi = (mode == Z_INV) ? z : bitrev(z, logN);
        buf[(f * TX + xl) * ls + zi] = v;
    }
    __syncthreads();
    if (mode != Z_INV) fft_dit(buf, N, logN, nf * TX, ls, tw, false);
    if (mode == Z_FWD_GAMMA_INV || mode == Z_FWD_RESID) {
        const bool apply = mode == Z_FWD_GAMMA_INV;
        T acc = (T)0;   // per-thread sum in the field precision; block and global sums in FP64
        for (int t = threadIdx.x; t < TX * N; t += blockDim.x) {
            const int kz = t / TX, xl = t - kz * TX;
            const int kx = kx0 + xl;
            if (kx >= Hx) continue;
            C s6[6];
            for (int f = 0; f < 6; ++f) s6[f] = buf[(f * TX + xl) * ls + kz];
            if (kx == 0 && ky == 0 && kz == 0 && mean6 != nullptr) {
                const double inv = 1.0 / ((double)N * N * N);
                for (int f = 0; f < 6; ++f) mean6[f] = (double)s6[f].x * inv;
            }
            const bool partner = !(kx == 0 || kx == (N >> 1));
            gamma_point<C, T>(s6, kx, ky, kz, N, lam0, mu0, acc, partner, apply);
            if (apply)
                for (int f = 0; f < 6; ++f) buf[(f * TX + xl) * ls + kz] = s6[f];
        }
        __syncthreads();
        const double tot = block_sum((double)acc, red);
        if (threadIdx.x == 0 && partials != nullptr) partials[blockIdx.x] = tot;
    }
    const bool fwd_only = mode == Z_FWD || mode == Z_FWD_RESID;
    if (!fwd_only) fft_dif(buf, N, logN, nf * TX, ls, tw, true);
    for (int t = threadIdx.x; t < nf * TX * N; t += blockDim.x) {
        const int f = t / (TX * N);
        const int r = t - f * TX * N;
        const int z = r / TX, xl = r - z * TX;
        const int kx = kx0 + xl;
        if (kx >= Hx) continue;
        const int zi = fwd_only ? z : bitrev(z, logN);
        spec[f * fstride + z * plane + (long)ky * Hx + kx] = buf[(f * TX + xl) * ls + zi];
    }
}

template <typename T> constexpr int tx_y() { return sizeof(T) == 4 ? 16 : 8; }
template <typename T> constexpr int tx_z() { return sizeof(T) == 4 ? 16 : 8; }

int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

int fft_z_blocks(int n, int is_double) {
    const int Hx = n / 2 + 1;
    const int TX = is_double ? tx_z<double>() : tx_z<float>();
    return n * ((Hx + TX - 1) / TX);
}

template <typename T>
cudaError_t fft_x_r2c(const T *in, void *spec, int n, int nfields, cudaStream_t s) {
    using C = typename CT<T>::type;
    const long npairs = (long)nfields * n * n / 2;
    const int blocks = (int)((npairs + kRowPairs - 1) / kRowPairs);
    const size_t sm = sizeof(C) * (n / 2 + (size_t)kRowPairs * n);
    k_fft_x_r2c<T><<<blocks, kThreads, sm, s>>>(in, (C *)spec, n, ilog2(n), npairs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fft_x_c2r(const void *spec, T *out, int n, int nfields, T scale, const double *add6,
                      cudaStream_t s) {
    using C = typename CT<T>::type;
    const long npairs = (long)nfields * n * n / 2;
    const int blocks = (int)((npairs + kRowPairs - 1) / kRowPairs);
    const size_t sm = sizeof(C) * (n / 2 + (size_t)kRowPairs * n);
    double a[6] = {0, 0, 0, 0, 0, 0};
    if (add6)
        for (int i = 0; i < 6; ++i) a[i] = add6[i];
    k_fft_x_c2r<T><<<blocks, kThreads, sm, s>>>((const C *)spec, out, n, ilog2(n), npairs, scale,
                                                add6 != nullptr, a[0], a[1], a[2], a[3], a[4], a[5]);
    return cudaGetLastError();
}

template <typename T> cudaError_t fft_y(void *spec, int n, int nfields, int inverse, cudaStream_t s) {
    using C = typename CT<T>::type;
    constexpr int TX = tx_y<T>();
    const int Hx = n / 2 + 1;
    const int blocks = nfields * n * ((Hx + TX - 1) / TX);
    const size_t sm = sizeof(C) * (n / 2 + (size_t)TX * (n + 1));
    k_fft_y<T, TX><<<blocks, kThreads, sm, s>>>((C *)spec, n, ilog2(n), inverse);
    return cudaGetLastError();
}

template <typename T>
cudaError_t fft_z(void *spec, int n, int nfields, int mode, double lam0, double mu0, double *partials,
                  double *mean6, cudaStream_t s) {
    using C = typename CT<T>::type;
    constexpr int TX = tx_z<T>();
    if ((mode == Z_FWD_GAMMA_INV || mode == Z_FWD_RESID) && nfields != 6) return cudaErrorInvalidValue;
    const int Hx = n / 2 + 1;
    const int blocks = n * ((Hx + TX - 1) / TX);
    const size_t sm = sizeof(C) * (n / 2 + (size_t)nfields * TX * (n + 1));
    static bool attr_set[2] = {false, false};
    if (!attr_set[sizeof(T) == 8]) {
        cudaError_t e = cudaFuncSetAttribute(k_fft_z<T, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[sizeof(T) == 8] = true;
    }
    if (sm > 220 * 1024) return cudaErrorInvalidValue;
    // one launch per group of fields that fits (nfields = 6 always fits for n <= 256)
    k_fft_z<T, TX><<<blocks, kThreads, sm, s>>>((C *)spec, n, ilog2(n), nfields, mode, (T)lam0,
                                                (T)mu0, partials, mean6);
    return cudaGetLastError();
}

template cudaError_t fft_x_r2c<float>(const float *, void *, int, int, cudaStream_t);
template cudaError_t fft_x_r2c<double>(const double *, void *, int, int, cudaStream_t);
template cudaError_t fft_x_c2r<float>(const void *, float *, int, int, float, const double *, cudaStream_t);
template cudaError_t fft_x_c2r<double>(const void *, double *, int, int, double, const double *, cudaStream_t);
template cudaError_t fft_y<float>(void *, int, int, int, cudaStream_t);
template cudaError_t fft_y<double>(void *, int, int, int, cudaStream_t);
template cudaError_t fft_z<float>(void *, int, int, int, double, double, double *, double *, cudaStream_t);
template cudaError_t fft_z<double>(void *, int, int, int, double, double, double *, double *, cudaStream_t);

}  // namespace evp
