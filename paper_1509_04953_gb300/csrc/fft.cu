// Hand-written 3D FFT passes for the Green-operator fixed point (Sec. 2.1: the spectral solve of
// the implicit stress update). One HBM round trip per axis:
//   x pass : real -> half spectrum, two real rows packed as one complex row
//   y pass : complex, lines along y loaded as [kx tile][y] (coalesced along kx)
//   z pass : complex, the six stress components of a [kx tile] x z slab of one ky; the forward
//            transform, the equilibrium residual, the Green-operator contraction and the inverse
//            transform run on the slab while it sits in shared memory
//   y pass : inverse
//   x pass : half spectrum -> real, fused with the strain update eps += field/N^3 + dE
// Where a (field, z) plane fits in shared memory next to two others, the x and y passes run as one launch
// per direction over whole planes (k_fft_xy_r2c, k_fft_xy_c2r), so an iteration crosses HBM three times.
// Spectra are [field][z|kz][ky][kx] with kx = 0..N/2 (row length N/2+1).
//
// Line transforms: Stockham auto-sort with register butterflies. N = R1 * R2 with R1 = min(N, 16)
// and R2 = N / R1 <= 16: a radix-R1 pass (no twiddles) and a radix-R2 pass (twiddles W_N^{r j}),
// natural order in and out. Shared-memory lines are padded (one slot per 16) so that the strided
// pass-1 writes hit distinct banks.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "common.cuh"
#include "fpctl.cuh"
#include "kernels.h"

namespace evp {

namespace {

constexpr int kThreads = 256;

// Asynchronous global -> shared copies (cp.async): every thread issues all of its loads before
// waiting, so many requests are in flight per SM while the pass is latency-bound.
template <int B> __device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (B == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else if constexpr (B == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
    else asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int N> struct Shape {
    static constexpr int R1 = N < 16 ? N : 16;
    static constexpr int R2 = N / R1;
    static constexpr int LS = N + N / 16 + 1;   // padded line stride
};
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <int L> struct Log2 { static constexpr int v = 1 + Log2<L / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

// cos(pi m / 8), m = 0..15: exact values of the sixteenth roots of unity.
__host__ __device__ constexpr double cos16(int m) {
    return m == 0 ? 1.0 : m == 1 ? 0.92387953251128675613 : m == 2 ? 0.70710678118654752440
         : m == 3 ? 0.38268343236508977173 : m == 4 ? 0.0 : m == 5 ? -0.38268343236508977173
         : m == 6 ? -0.70710678118654752440 : m == 7 ? -0.92387953251128675613 : m == 8 ? -1.0
         : m == 9 ? -0.92387953251128675613 : m == 10 ? -0.70710678118654752440
         : m == 11 ? -0.38268343236508977173 : m == 12 ? 0.0 : m == 13 ? 0.38268343236508977173
         : m == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}

template <int M> __host__ __device__ constexpr int brev_c(int i) {
    int r = 0;
    for (int b = 0; b < M; ++b) r |= ((i >> b) & 1) << (M - 1 - b);
    return r;
}

// Length-R DFT of x held in registers (radix-2 network with constant twiddles). The forward
// twiddle W_{2h}^p = exp(-2 pi i p / 2h) = (cos(pi m/8), -sin(pi m/8)), m = 16 p / 2h, with
// sin(pi m/8) = cos(pi (m + 12)/8). INV uses the conjugate. The twiddles 1 (m = 0) and -i (m = 4; +i inverse)
// are applied as a copy and a swap with a sign change: without fast-math the compiler keeps the products by
// the zero component, and these are 22 of the 32 twiddles of a 16-point DFT (10 of 12 at 8 points).
template <int R, bool INV, typename C> __device__ __forceinline__ void dft_reg(C (&x)[R]) {
    using T = decltype(C::x);
    constexpr int LR = Log2<R>::v;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = brev_c<LR>(i);
        if (j > i) { const C t = x[i]; x[i] = x[j]; x[j] = t; }
    }
#pragma unroll
    for (int h = 1; h < R; h <<= 1) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * h) {
#pragma unroll
            for (int p = 0; p < h; ++p) {
                const int m = p * (16 / (2 * h));
                const C b0 = x[g + p + h];
                C b;
                if (m == 0) {
                    b = b0;
                } else if (m == 4) {
                    b = INV ? cmk<C>(-b0.y, b0.x) : cmk<C>(b0.y, -b0.x);
                } else {
                    const T wc = (T)cos16(m);
                    const T ws = INV ? (T)cos16((m + 12) & 15) : -(T)cos16((m + 12) & 15);
                    b = cmk<C>(b0.x * wc - b0.y * ws, b0.x * ws + b0.y * wc);
                }
                const C a = x[g + p];
                x[g + p] = cadd(a, b);
                x[g + p + h] = csub(a, b);
            }
        }
    }
}

// Item t of the radix-R1 pass -> (line l, j < M1). With M1 = 8 (N = 128) a half-warp spans two lines of 8 items;
// lines l and l + 1 lie 2 LS = 18 banks apart (mod 32) and share a bank pair, lines l and l + 8 lie 16 apart and
// share none. So within each group of 16 lines the half-warps take lines (l, l + 8); the lines past the last full
// group keep the plain order. Any mapping of items to threads gives the same values.
template <int N> __device__ __forceinline__ void pass1_item(int t, int nlines, int &l, int &j) {
    constexpr int M1 = N / Shape<N>::R1;
    if constexpr (M1 == 8 && Shape<N>::LS % 16 == 9) {
        if (t < (nlines >> 4) * 16 * M1) {
            const int hw = t >> 4, lane = t & 15;
            l = ((hw >> 3) << 4) + (hw & 7) + ((lane >> 3) << 3);
            j = lane & 7;
            return;
        }
    }
    l = t / M1;
    j = t - l * M1;
}

// Element r of a z-pass slab -> (z, column xl < TX) for the column loads, the Green-operator phase and the
// stores. With TX = 8 a half-warp spans 8 columns of two planes; planes z and z + 1 put columns 0 and 7 on one bank
// pair (line stride LS = 9 mod 16), planes z and z + 8 (in one 16-plane block) share none. Global accesses keep
// 8 consecutive columns of a plane per half-warp row.
template <int N, int TX> __device__ __forceinline__ void slab_item(int r, int &z, int &xl) {
    if constexpr (TX == 8 && N % 16 == 0 && Shape<N>::LS % 16 == 9) {
        const int hw = r >> 4, lane = r & 15;
        z = ((hw >> 3) << 4) + (hw & 7) + ((lane >> 3) << 3);
        xl = lane & 7;
    } else {
        z = r / TX;
        xl = r % TX;
    }
}

// The two passes of block_fft (R2 > 1), also called on their own by the z pass.
// pass 1: radix R1, Ns = 1: item (l, j < M1) reads slots j + M1 r and writes j R1 + r, so
// every read completes before any write (held in registers across a barrier). With j < M1 and M1 | 16
// the padded slots are pad16(j + M1 r) = j + pad16(M1 r) and pad16(16 j + r) = 17 j + r (r < 16): one base
// address per item and compile-time offsets. Ends with a barrier.
template <int N, bool INV, int MAXIT, typename C> __device__ void bfft_pass1(C *buf, int nlines) {
    constexpr int R1 = Shape<N>::R1, LS = Shape<N>::LS;
    constexpr int M1 = N / R1;
    static_assert(16 % M1 == 0 || M1 % 16 == 0, "pass-1 stride");
    const int items = nlines * M1;
    C v[MAXIT][R1];
#pragma unroll
    for (int it = 0; it < MAXIT; ++it) {
        const int t = threadIdx.x + it * blockDim.x;
        if (t < items) {
            int l, j;
            pass1_item<N>(t, nlines, l, j);
            const C *src = buf + l * LS + (M1 <= 16 ? j : pad16(j));
#pragma unroll
            for (int r = 0; r < R1; ++r) v[it][r] = src[M1 <= 16 ? pad16(r * M1) : r * (M1 + M1 / 16)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < MAXIT; ++it) {
        const int t = threadIdx.x + it * blockDim.x;
        if (t < items) {
            int l, j;
            pass1_item<N>(t, nlines, l, j);
            dft_reg<R1, INV>(v[it]);
            C *dst = buf + l * LS + 17 * j;
#pragma unroll
            for (int r = 0; r < R1; ++r) dst[r] = v[it][r];
        }
    }
    __syncthreads();
}

// pass 2: radix R2, Ns = R1 = 16: item (l, j < 16) reads and writes slots j + 16 r only, which are
// pad16(j + 16 r) = j + 17 r
// Every CTA has a multiple of 16 threads, so a thread's items share one j = threadIdx.x mod 16 and its
// twiddles tw[16 r + j] = exp(-2 pi i r j / N) are loaded once, into registers. Ends with a barrier.
template <int N, bool INV, typename C> __device__ void bfft_pass2(C *buf, int nlines, const C *tw) {
    constexpr int R2 = Shape<N>::R2, LS = Shape<N>::LS;
    const int jt = threadIdx.x & 15;
    C wr[R2];
#pragma unroll
    for (int r = 1; r < R2; ++r) {
        wr[r] = tw[16 * r + jt];   // r-major: a half-warp reads 16 in a row
        if (INV) wr[r].y = -wr[r].y;
    }
    for (int t = threadIdx.x; t < nlines * 16; t += blockDim.x) {
        const int l = t >> 4;
        C *line = buf + l * LS + jt;
        C u[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            C a = line[17 * r];
            if (r > 0) a = cmul(a, wr[r]);
            u[r] = a;
        }
        dft_reg<R2, INV>(u);
#pragma unroll
        for (int r = 0; r < R2; ++r) line[17 * r] = u[r];
    }
    __syncthreads();
}

// In-place transform of nlines padded lines (line l at buf + l*LS). tw[16 r + j] = exp(-2 pi i r j / N)
// (see load_tw),
// m < N. Starts after and ends with a barrier. MAXIT >= ceil(nlines * (N/R1) / blockDim).
template <int N, bool INV, int MAXIT, typename C> __device__ void block_fft(C *buf, int nlines, const C *tw) {
    constexpr int R1 = Shape<N>::R1, R2 = Shape<N>::R2, LS = Shape<N>::LS;
    if constexpr (R2 == 1) {   // a single radix-N pass; every line is owned by one thread
        for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
            C v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = buf[l * LS + pad16(r)];
            dft_reg<R1, INV>(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) buf[l * LS + pad16(r)] = v[r];
        }
        __syncthreads();
    } else {
        bfft_pass1<N, INV, MAXIT>(buf, nlines);
        bfft_pass2<N, INV>(buf, nlines, tw);
    }
}

// Twiddles of the radix-R2 pass, computed once per CTA into shared memory in the precision of the transform
// (the FP64 pipe is 1/58 of the FP32 rate on this GPU, so FP32 transforms avoid it): slot k = 16 r + j holds
// exp(-2 pi i r j / N) for r < N/16, j < 16 (r j < N), so the 16 lanes of a half-warp, which differ in j, read
// 16 consecutive slots (indexed by the product r j the stride-r reads hit the same banks).
__device__ __forceinline__ void load_tw(float2 *tw_s, int N) {
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        float sn, cs;
        sincospif(-2.0f * (float)((k >> 4) * (k & 15)) / (float)N, &sn, &cs);
        tw_s[k] = make_float2(cs, sn);
    }
}
__device__ __forceinline__ void load_tw(double2 *tw_s, int N) {
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)((k >> 4) * (k & 15)) / (double)N, &sn, &cs);
        tw_s[k] = make_double2(cs, sn);
    }
}

template <int N> __host__ __device__ constexpr int rowpairs() { return N >= 64 ? 32 : 4096 / (N * 2); }
// Column tiles of the half spectrum (kx = 0..N/2): N/2 columns split into full tiles of TXe, and the
// Nyquist column kx = N/2 appended to tile 0 as one extra line, so no tile is ragged.
template <int N, typename T> __host__ __device__ constexpr int tx_y() {
    return (sizeof(T) == 4 ? 32 : 16) < N / 2 ? (sizeof(T) == 4 ? 32 : 16) : N / 2;
}
template <int N, typename T> __host__ __device__ constexpr int tx_z() {
    return (sizeof(T) == 4 ? 8 : 4) < N / 2 ? (sizeof(T) == 4 ? 8 : 4) : N / 2;
}
template <int N> __host__ __device__ constexpr int maxit(int lines, int threads = kThreads) {
    return (lines * (N / Shape<N>::R1) + threads - 1) / threads < 1 ? 1
                                                                   : (lines * (N / Shape<N>::R1) + threads - 1) / threads;
}
// Threads of a column-tile CTA: enough that a tile with its extra Nyquist lines (lines + extra)
// needs no more pass-1 register sets than a full tile would at kThreads (the extra set would raise
// register use, and so cut occupancy, for every tile).
template <int N> __host__ __device__ constexpr int tile_threads(int lines, int extra) {
    return ((((lines + extra) * (N / Shape<N>::R1) + maxit<N>(lines) - 1) / maxit<N>(lines) + 31) / 32) * 32 < kThreads
               ? kThreads
               : ((((lines + extra) * (N / Shape<N>::R1) + maxit<N>(lines) - 1) / maxit<N>(lines) + 31) / 32) * 32;
}
template <int N, typename T> __host__ __device__ constexpr int y_threads() { return tile_threads<N>(tx_y<N, T>(), 1); }
template <int N, typename T> __host__ __device__ constexpr int z_threads() { return tile_threads<N>(6 * tx_z<N, T>(), 6); }

// ---------------------------------------------------------------------------------------------
// x pass, real -> half spectrum. CTA = RP pairs of rows (y even, y+1) of one (field, z).
// ---------------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(kThreads, N >= 64 && N <= 128 ? (sizeof(T) == 4 ? 6 : 3) : 1) k_fft_x_r2c(const T *__restrict__ in, typename CT<T>::type *__restrict__ out,
                                                       long npairs, const int *__restrict__ skip) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    using C = typename CT<T>::type;
    constexpr int RP = rowpairs<N>(), LS = Shape<N>::LS, Hx = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + N;
    load_tw(tw, N);
    const long p0 = (long)blockIdx.x * RP;
    const int np = (int)min((long)RP, npairs - p0);
    for (int t = threadIdx.x; t < np * N; t += blockDim.x) {
        const int pl = t / N, j = t - pl * N;
        const long row0 = 2 * (p0 + pl);            // global row index = (field*N + z)*N + y
        T *slot = reinterpret_cast<T *>(buf + pl * LS + pad16(j));
        cp_async<sizeof(T)>(slot, in + row0 * N + j);
        cp_async<sizeof(T)>(slot + 1, in + (row0 + 1) * N + j);
    }
    cp_async_wait_all();
    __syncthreads();
    block_fft<N, false, maxit<N>(RP)>(buf, np, tw);
    const T h = (T)0.5;
    for (int t = threadIdx.x; t < np * Hx; t += blockDim.x) {
        const int pl = t / Hx, k = t - pl * Hx;
        const C zk = buf[pl * LS + pad16(k & (N - 1))];
        const C zc = cconj(buf[pl * LS + pad16((N - k) & (N - 1))]);
        const long row0 = 2 * (p0 + pl);
        out[row0 * Hx + k] = cmk<C>(h * (zk.x + zc.x), h * (zk.y + zc.y));
        out[(row0 + 1) * Hx + k] = cmk<C>(h * (zk.y - zc.y), -h * (zk.x - zc.x));   // (zk - zc) / 2i
    }
}

// ---------------------------------------------------------------------------------------------
// x pass, half spectrum -> real (complex-to-real through the same row-pair packing). The CTA's rows
// are contiguous in both the half spectrum and the strain, so both arrive by 16-byte asynchronous
// copies into shared memory before the transform; every global access is then a wide, coalesced one.
// ---------------------------------------------------------------------------------------------
template <int N> __host__ __device__ constexpr int rowpairs_c2r() { return rowpairs<N>() > 16 ? 16 : rowpairs<N>(); }

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_fft_x_c2r(const typename CT<T>::type *__restrict__ spec, T *__restrict__ out,
                                                       long npairs, T scale, int has_add, T a0, T a1, T a2, T a3, T a4,
                                                       T a5, const T *__restrict__ base, const int *__restrict__ skip) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    using C = typename CT<T>::type;
    constexpr int RP = rowpairs_c2r<N>(), LS = Shape<N>::LS, Hx = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + N;                          // RP packed lines
    C *hs = buf + RP * LS;                    // 2 RP half-spectrum rows, row-major
    T *bs = reinterpret_cast<T *>(hs + 2 * RP * Hx);   // 2 RP strain rows (with has_add)
    const long p0 = (long)blockIdx.x * RP;
    const int np = (int)min((long)RP, npairs - p0);
    {   // rows 2 p0 .. 2 (p0 + np) - 1: contiguous, 16-byte aligned (2 Hx sizeof(C) and 2 N sizeof(T) are)
        const uint4 *src = reinterpret_cast<const uint4 *>(spec + 2 * p0 * Hx);
        uint4 *dst = reinterpret_cast<uint4 *>(hs);
        const int nchunk = (int)(2 * np * Hx * sizeof(C) / 16);
        for (int t = threadIdx.x; t < nchunk; t += blockDim.x) cp_async<16>(dst + t, src + t);
        if (has_add) {
            const T *bsrc = base ? base : out;
            const uint4 *src2 = reinterpret_cast<const uint4 *>(bsrc + 2 * p0 * N);
            uint4 *dst2 = reinterpret_cast<uint4 *>(bs);
            const int nchunk2 = (int)(2 * np * N * sizeof(T) / 16);
            for (int t = threadIdx.x; t < nchunk2; t += blockDim.x) cp_async<16>(dst2 + t, src2 + t);
        }
    }
    load_tw(tw, N);
    cp_async_wait_all();
    __syncthreads();
    for (int t = threadIdx.x; t < np * N; t += blockDim.x) {
        const int pl = t / N, k = t - pl * N;
        const C *ra = hs + 2 * pl * Hx, *rb = ra + Hx;
        C A, B;
        if (k <= (N >> 1)) {
            A = ra[k];
            B = rb[k];
        } else {
            A = cconj(ra[N - k]);
            B = cconj(rb[N - k]);
        }
        buf[pl * LS + pad16(k)] = cmk<C>(A.x - B.y, A.y + B.x);   // A + iB
    }
    __syncthreads();
    block_fft<N, true, maxit<N>(RP)>(buf, np, tw);
    const long rows_per_field = (long)N * N;
    for (int t = threadIdx.x; t < np * N; t += blockDim.x) {
        const int pl = t / N, j = t - pl * N;
        const long row0 = 2 * (p0 + pl);
        const C z = buf[pl * LS + pad16(j)];
        if (has_add) {
            const int f = (int)(row0 / rows_per_field);
            const T add = f == 0 ? a0 : f == 1 ? a1 : f == 2 ? a2 : f == 3 ? a3 : f == 4 ? a4 : a5;
            out[row0 * N + j] = bs[2 * pl * N + j] + (z.x * scale + add);
            out[(row0 + 1) * N + j] = bs[(2 * pl + 1) * N + j] + (z.y * scale + add);
        } else {
            out[row0 * N + j] = z.x;
            out[(row0 + 1) * N + j] = z.y;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// y pass: CTA = (field, z, kx tile of TX columns); lines along y.
// ---------------------------------------------------------------------------------------------
template <typename T, int N, bool INV>
__global__ void __launch_bounds__(y_threads<N, T>(), sizeof(T) == 4 && N >= 64 && N <= 128 ? 5 : 1)
k_fft_y(typename CT<T>::type *__restrict__ spec, const int *__restrict__ skip) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    using C = typename CT<T>::type;
    constexpr int TX = tx_y<N, T>(), LS = Shape<N>::LS, Hx = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + N;
    constexpr int ntiles = (N / 2) / TX;
    const int tile = blockIdx.x % ntiles;
    const long plane = blockIdx.x / ntiles;        // field*N + z
    const bool nyq = tile == 0;                    // tile 0 also carries the column kx = N/2 as line TX
    C *base = spec + plane * (long)N * Hx;
    const int kx0 = tile * TX;
    load_tw(tw, N);
    for (int t = threadIdx.x; t < TX * N; t += blockDim.x) {   // TX, N powers of two: shifts, no division
        const int y = t / TX, xl = t % TX;
        cp_async<sizeof(C)>(buf + xl * LS + pad16(y), base + (long)y * Hx + kx0 + xl);
    }
    if (nyq)
        for (int y = threadIdx.x; y < N; y += blockDim.x)
            cp_async<sizeof(C)>(buf + TX * LS + pad16(y), base + (long)y * Hx + N / 2);
    cp_async_wait_all();
    __syncthreads();
    block_fft<N, INV, maxit<N>(TX + 1, y_threads<N, T>())>(buf, TX + (nyq ? 1 : 0), tw);
    for (int t = threadIdx.x; t < TX * N; t += blockDim.x) {
        const int y = t / TX, xl = t % TX;
        base[(long)y * Hx + kx0 + xl] = buf[xl * LS + pad16(y)];
    }
    if (nyq)
        for (int y = threadIdx.x; y < N; y += blockDim.x) base[(long)y * Hx + N / 2] = buf[TX * LS + pad16(y)];
}

// ---------------------------------------------------------------------------------------------
// x and y passes fused: CTA = one (field, z) plane held in shared memory. The x transform runs on
// N/2 packed row pairs (line p = rows 2p, 2p+1, as in the x pass); the half-spectrum rows then replace
// their line in place (row 2p at slots 0..N/2 of line p, row 2p+1 at slots N/2+1..N+1), and the y
// transform runs down the N/2+1 columns of that row-major plane. Every value goes through the same
// operations, in the same order, as in the separate x and y passes, so the spectra are bitwise the same;
// the plane crosses HBM once instead of twice. Used where the plane fits (xy_fused).
// ---------------------------------------------------------------------------------------------
// One thread per pass-1 item of the N/2 row-pair lines (x) and of the N/2 regular columns (y); the Nyquist
// column's few pass-1 items run on lanes of warp 0 (col_pass1).
template <int N> __host__ __device__ constexpr int xy_threads() {
    return (((N / 2) * (N / Shape<N>::R1) + 31) / 32) * 32;
}
template <typename T, int N> __host__ __device__ constexpr size_t smem_xy() {
    return sizeof(typename CT<T>::type) * (N + (size_t)(N / 2) * Shape<N>::LS);
}
// The plane fits next to two others on one SM (FP32 up to N = 128, FP64 up to N = 64), the row pair of the
// half spectrum fits in a padded line (2 (N/2+1) <= LS), and both passes are two-radix Stockham passes.
template <typename T, int N> __host__ __device__ constexpr bool xy_fused() {
    return N >= 32 && Shape<N>::R2 > 1 && 2 * (N / 2 + 1) <= Shape<N>::LS && smem_xy<T, N>() <= 72 * 1024;
}
template <typename T, int N> __host__ __device__ constexpr int xy_ctas() {
    return sizeof(T) == 4 ? (N >= 128 ? 3 : N == 64 ? 8 : 1) : 1;
}

// Slot of half-spectrum row y, column kx in the row-major plane (rows 2p and 2p+1 share line p).
template <int N> __device__ __forceinline__ int xy_at(int y, int kx) {
    return (y >> 1) * Shape<N>::LS + (y & 1) * (N / 2 + 1) + kx;
}

// The passes of the plane transforms, one pass-1 item per thread (blockDim.x >= items). Each has the items,
// operands and twiddles of block_fft's passes (x: lines of the packed row pairs) or of the y pass (columns,
// addressed through xy_at, kx-fastest so a warp touches consecutive slots); only where the values come from
// or go to differs: the first pass of the forward kernel reads HBM straight into registers, and so do the
// inverse kernel's first pass and the forward kernel's last pass store, so none of them round-trips through
// shared memory.

// x pass 1 (bfft_pass1's items) with element e of line l read through ld(l, e). IN_PLACE: ld reads the lines the
// pass writes, so every read comes before any write (a barrier between); otherwise it reads HBM. Ends with a barrier.
template <int N, bool INV, bool IN_PLACE, typename C, typename Ld> __device__ void x_pass1_ld(C *buf, int nlines, Ld ld) {
    constexpr int R1 = Shape<N>::R1, LS = Shape<N>::LS, M1 = N / R1;
    static_assert(M1 <= 16 && 16 % M1 == 0, "pass-1 stride");
    const int t = threadIdx.x;
    const bool on = t < nlines * M1;
    int l = 0, j = 0;
    if (on) pass1_item<N>(t, nlines, l, j);
    C v[R1];
    if (on) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = ld(l, j + M1 * r);
    }
    if constexpr (IN_PLACE) __syncthreads();
    if (on) {
        dft_reg<R1, INV>(v);
        C *dst = buf + l * LS + 17 * j;
#pragma unroll
        for (int r = 0; r < R1; ++r) dst[r] = v[r];
    }
    __syncthreads();
}

// y pass 1: item (kx, j < M1) takes rows j + M1 r of column kx through ld(y, kx) and writes rows R1 j + r (line
// R1 j / 2 + r / 2, half r & 1). IN_PLACE: ld reads the buffer the pass writes, so every read comes before any write
// (a barrier between). The regular columns kx < N/2 take one item per thread; the Nyquist column's M1 items then run
// on lanes 0..M1-1 of warp 0 (no other item writes that column), reading its rows through ldn(y), which must not
// read what the regular items write (pre(), run by every thread in the read phase, could copy them aside); a warp
// barrier orders those lanes' reads before their in-place writes. Ends with a barrier.
template <int N, bool INV, bool IN_PLACE, typename C, typename Ld, typename Pre, typename LdN>
__device__ void col_pass1(C *buf, Ld ld, Pre pre, LdN ldn) {
    constexpr int R1 = Shape<N>::R1, M1 = N / R1, Hx = N / 2 + 1, LS = Shape<N>::LS;
    static_assert(M1 % 2 == 0 && R1 % 2 == 0 && M1 <= 32, "row pairs");
    auto transform = [&](int j, int kx, C (&v)[R1]) {
        dft_reg<R1, INV>(v);
        C *dst = buf + (R1 / 2) * j * LS + kx;
#pragma unroll
        for (int r = 0; r < R1; ++r) dst[(r >> 1) * LS + (r & 1) * Hx] = v[r];
    };
    const int t = threadIdx.x;
    const bool on = t < (N / 2) * M1;
    const int j = t / (N / 2), kx = t % (N / 2);
    C v[R1];
    if (on) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = ld(j + M1 * r, kx);
    }
    pre();
    if constexpr (IN_PLACE) __syncthreads();
    if (on) transform(j, kx, v);
    if (t < M1) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = ldn(t + M1 * r);
        __syncwarp((1u << M1) - 1u);   // ldn may read the column these lanes write
        transform(t, N / 2, v);
    }
    __syncthreads();
}

// y pass 2: item (kx, j < 16) transforms rows j + 16 r (line (j >> 1) + 8 r, half j & 1) and hands its outputs
// (row j + 16 r in u[r]) to st(j, kx, slot of row j, u). Ends with a barrier.
template <int N, bool INV, typename C, typename St> __device__ void col_pass2(C *buf, const C *tw, St st) {
    constexpr int R1 = Shape<N>::R1, R2 = Shape<N>::R2, Hx = N / 2 + 1, LS = Shape<N>::LS;
    for (int t = threadIdx.x; t < Hx * R1; t += blockDim.x) {
        const int j = t / Hx, kx = t - j * Hx;
        C *line = buf + xy_at<N>(j, kx);
        C u[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            C a = line[r * (R1 / 2) * LS];
            if (r > 0) {
                C w = tw[16 * r + j];
                if (INV) w.y = -w.y;
                a = cmul(a, w);
            }
            u[r] = a;
        }
        dft_reg<R2, INV>(u);
        st(j, kx, line, u);
    }
    __syncthreads();
}

template <typename T, int N>
__global__ void __launch_bounds__(xy_threads<N>(), xy_ctas<T, N>())
k_fft_xy_r2c(const T *__restrict__ in, typename CT<T>::type *__restrict__ out, const int *__restrict__ skip) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    using C = typename CT<T>::type;
    constexpr int LS = Shape<N>::LS, Hx = N / 2 + 1, NP = N / 2, KU = (Hx + 31) / 32, R2 = Shape<N>::R2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + N;
    const T *src = in + (long)blockIdx.x * N * N;   // plane = field * N + z
    C *dst = out + (long)blockIdx.x * N * Hx;
    load_tw(tw, N);
    // x: line p packs rows 2p and 2p+1 as one complex row; pass 1 reads them from HBM
    x_pass1_ld<N, false, false>(buf, NP, [&](int p, int e) { return cmk<C>(src[(2 * p) * N + e], src[(2 * p + 1) * N + e]); });
    bfft_pass2<N, false>(buf, NP, tw);
    {   // unpack one line per warp: read the line's values, then write its two half-spectrum rows in place
        const int lane = threadIdx.x & 31;
        const T h = (T)0.5;
        for (int p = threadIdx.x >> 5; p < NP; p += blockDim.x >> 5) {
            C *line = buf + p * LS;
            C a[KU], b[KU];
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                const int k = lane + 32 * u;
                if (k < Hx) {
                    const C zk = line[pad16(k & (N - 1))];
                    const C zc = cconj(line[pad16((N - k) & (N - 1))]);
                    a[u] = cmk<C>(h * (zk.x + zc.x), h * (zk.y + zc.y));
                    b[u] = cmk<C>(h * (zk.y - zc.y), -h * (zk.x - zc.x));   // (zk - zc) / 2i
                }
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                const int k = lane + 32 * u;
                if (k < Hx) {
                    line[k] = a[u];
                    line[Hx + k] = b[u];
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // y: down the columns of the row-major plane; pass 2 stores rows j + 16 r to HBM
    // y: down the columns of the row-major plane; pass 2 stores rows j + 16 r to HBM
    col_pass1<N, false, true>(
        buf, [&](int y, int kx) { return buf[xy_at<N>(y, kx)]; }, [] {}, [&](int y) { return buf[xy_at<N>(y, N / 2)]; });
    col_pass2<N, false>(buf, tw, [&](int j, int kx, C *, const C (&u)[R2]) {
#pragma unroll
        for (int r = 0; r < R2; ++r) dst[(j + 16 * r) * Hx + kx] = u[r];
    });
}

// The inverse: y transform down the columns, the row pairs packed as one complex line (A + iB), the x
// transform, and the strain update of the x pass's epilogue.
template <typename T, int N>
__global__ void __launch_bounds__(xy_threads<N>(), xy_ctas<T, N>())
k_fft_xy_c2r(const typename CT<T>::type *__restrict__ spec, T *__restrict__ out, T scale, int has_add, T a0, T a1, T a2,
             T a3, T a4, T a5, const T *__restrict__ base, const int *__restrict__ skip) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    using C = typename CT<T>::type;
    constexpr int LS = Shape<N>::LS, Hx = N / 2 + 1, NP = N / 2, R2 = Shape<N>::R2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + N;
    const C *src = spec + (long)blockIdx.x * N * Hx;
    load_tw(tw, N);
    // y: pass 1 reads the columns from HBM
    col_pass1<N, true, false>(
        buf, [&](int y, int kx) { return src[y * Hx + kx]; }, [] {}, [&](int y) { return src[y * Hx + N / 2]; });
    col_pass2<N, true>(buf, tw, [](int, int, C *line, const C (&u)[R2]) {
#pragma unroll
        for (int r = 0; r < R2; ++r) line[r * 8 * LS] = u[r];
    });
    // x: pass 1 packs rows 2p and 2p+1 as it reads them (Z[k] = A[k] + i B[k], with A[N-k] = conj A[k] past N/2)
    // and writes the lines in place
    x_pass1_ld<N, true, true>(buf, NP, [&](int p, int k) {
        const C *line = buf + p * LS;
        C A, B;
        if (k <= (N >> 1)) {
            A = line[k];
            B = line[Hx + k];
        } else {
            A = cconj(line[N - k]);
            B = cconj(line[Hx + N - k]);
        }
        return cmk<C>(A.x - B.y, A.y + B.x);
    });
    bfft_pass2<N, true>(buf, NP, tw);
    const long r0 = (long)blockIdx.x * N;   // first row: (field * N + z) * N
    T add = (T)0;
    if (has_add) {
        const int f = (int)(blockIdx.x / N);
        add = f == 0 ? a0 : f == 1 ? a1 : f == 2 ? a2 : f == 3 ? a3 : f == 4 ? a4 : a5;
    }
    const T *bsrc = base ? base : out;
    for (int t = threadIdx.x; t < NP * N; t += blockDim.x) {
        const int p = t / N, j = t - p * N;
        const C z = buf[p * LS + pad16(j)];
        const long o0 = (r0 + 2 * p) * N + j, o1 = o0 + N;
        if (has_add) {
            out[o0] = bsrc[o0] + (z.x * scale + add);
            out[o1] = bsrc[o1] + (z.y * scale + add);
        } else {
            out[o0] = z.x;
            out[o1] = z.y;
        }
    }
}

// Green operator of the isotropic reference medium applied to one spectral stress (Mandel):
// eps_kh = (n_h v_k + n_k v_h)/(2 mu0) - c n_k n_h (n.v), v = sigma.n, n = xi/|xi|,
// c = (lam0+mu0)/(mu0 (lam0+2 mu0)). At frequencies with a Nyquist component the compliance of
// the reference medium replaces it; the zero frequency is left to the macroscopic update.
// Returns -Gamma:sigma in s (in place) if apply, and accumulates |xi.sigma|^2 (xi = 2 pi k/N).
template <typename C, typename T>
__device__ __forceinline__ void gamma_point(C s[6], int kx, int ky, int kz, int N, T lam0, T mu0, T &acc, bool partner,
                                            bool apply) {
    const int fx = kx;                                   // 0..N/2
    const int fy = ky <= (N >> 1) ? ky : ky - N;
    const int fz = kz <= (N >> 1) ? kz : kz - N;
    const T r2 = (T)0.70710678118654752440;
    const C t11 = s[0], t22 = s[1], t33 = s[2];
    const C t23 = cmk<C>(s[3].x * r2, s[3].y * r2), t13 = cmk<C>(s[4].x * r2, s[4].y * r2),
            t12 = cmk<C>(s[5].x * r2, s[5].y * r2);
    const int h = N >> 1;
    const bool nyq = kx == h || ky == h || kz == h;
    // Where the Green operator is applied (not on a Nyquist plane, not at zero frequency) the residual comes from
    // its v = sigma_hat n: |xi.sigma_hat|^2 = w^2 |f|^2 |v|^2, the same at the Hermitian partner -k
    const bool fused = apply && !nyq && !(fx == 0 && fy == 0 && fz == 0);
    if (!fused) {   // equilibrium residual |xi.sigma_hat|^2 at this frequency and, for 0 < kx < N/2, at its
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
    if (nyq) {
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
    {   // the residual of this frequency (and of its partner, counted twice)
        const T w = (T)(6.283185307179586476925 / N);
        const T f2 = (T)(fx * fx + fy * fy + fz * fz);
        const T vv = v1.x * v1.x + v1.y * v1.y + v2.x * v2.x + v2.y * v2.y + v3.x * v3.x + v3.y * v3.y;
        acc += (partner ? (T)2 : (T)1) * (w * w * f2) * vv;
    }
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
template <typename T, int N>
__global__ void __launch_bounds__(z_threads<N, T>(), sizeof(T) == 4 && N <= 128 ? 3 : 1) k_fft_z(typename CT<T>::type *__restrict__ spec, int nf, int mode, T lam0,
                                                   T mu0, double *__restrict__ partials, double *__restrict__ mean6, const int *__restrict__ skip,
                                                   ZCtl zc) {
    pdl_wait();
    pdl_trigger();
    if (skip != nullptr && *skip) return;   // the fixed point has converged
    using C = typename CT<T>::type;
    constexpr int TX = tx_z<N, T>(), LS = Shape<N>::LS, Hx = N / 2 + 1, MI = maxit<N>(6 * (TX + 1), z_threads<N, T>());
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *tw = reinterpret_cast<C *>(smem_raw);
    C *buf = tw + N;
    __shared__ double red[32];
    constexpr int ntiles = (N / 2) / TX;
    const int tile = blockIdx.x % ntiles;
    const int ky = blockIdx.x / ntiles;
    // lines: f*TX + xl for the TX regular columns of field f, then (tile 0 only) nf*TX + f for the
    // Nyquist column kx = N/2 of field f
    const bool nyq = tile == 0;
    const int kx0 = tile * TX;
    const int nlines = nf * TX + (nyq ? nf : 0);
    const long plane = (long)N * Hx;            // one z plane of one field
    const long fstride = plane * N;
    load_tw(tw, N);
    // The slab walk: element r = t mod (TX N) of field f sits at column xl and plane z = slab_item(r). With
    // NT threads and NT | TX N, a thread keeps its column, and its planes advance by DZ = NT / TX per step
    // (slab_item adds DZ to z when r grows by NT, and pad16 adds DZ + DZ / 16 when DZ is a multiple of 16), so its
    // shared and global addresses advance by constant strides.
    constexpr int NT = z_threads<N, T>(), DZ = NT / TX, KZ = TX * N / NT;
    constexpr bool walk = (TX * N) % NT == 0 && DZ % 16 == 0 &&
                          ((TX == 8 && N % 16 == 0 && LS % 16 == 9) ? NT % 128 == 0 : NT % TX == 0);
    int wz = 0, wxl = 0;
    if constexpr (walk) slab_item<N, TX>((int)threadIdx.x, wz, wxl);
    // Item it of an HBM-side step over the slab's lines with L items per line: regular lines (field f, column
    // xl) take it = (f L + i) TX + xl, xl fastest, so 8 lanes touch 8 consecutive columns of one plane; the Nyquist
    // lines (tile 0) follow. Gives the line, the item's index i < L and the column's first element in HBM.
    auto hbm_item = [&](int it, int L, int &l, int &i) -> C * {
        const int nreg = nf * TX * L;
        if (it < nreg) {
            const int xl = it % TX, f = it / (TX * L);
            i = (it / TX) % L;
            l = f * TX + xl;
            return spec + f * fstride + (long)ky * Hx + kx0 + xl;
        }
        const int q = it - nreg, f = q / L;
        i = q - f * L;
        l = nf * TX + f;
        return spec + f * fstride + (long)ky * Hx + N / 2;
    };
    if (mode != Z_INV) {
        // the forward transform's pass 1 (the whole transform when R2 = 1) straight from HBM: item (line, j < M1)
        // reads elements j + M1 r and writes slots 16 j + r (slot r when R2 = 1), as bfft_pass1
        constexpr int R1 = Shape<N>::R1, M1 = N / R1;
        const int nit = nlines * M1;
        for (int it = threadIdx.x; it < nit; it += blockDim.x) {
            int l, j;
            const C *g = hbm_item(it, M1, l, j);
            C v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = g[(long)(j + M1 * r) * plane];
            dft_reg<R1, false>(v);
            C *dst = buf + l * LS + 17 * j;
#pragma unroll
            for (int r = 0; r < R1; ++r) dst[r] = v[r];
        }
        __syncthreads();
        if constexpr (Shape<N>::R2 > 1) bfft_pass2<N, false>(buf, nlines, tw);
    } else {
        if constexpr (walk) {
            C *sb = buf + wxl * LS + pad16(wz);
            const C *gb = spec + (long)wz * plane + (long)ky * Hx + kx0 + wxl;
            for (int f = 0; f < nf; ++f) {
#pragma unroll
                for (int k = 0; k < KZ; ++k)
                    cp_async<sizeof(C)>(sb + f * TX * LS + k * (DZ + DZ / 16), gb + f * fstride + (long)k * DZ * plane);
            }
        } else {
            for (int t = threadIdx.x; t < nf * TX * N; t += blockDim.x) {   // TX, N powers of two: shifts
                const int f = t / (TX * N), r = t % (TX * N);
                int z, xl;
                slab_item<N, TX>(r, z, xl);
                cp_async<sizeof(C)>(buf + (f * TX + xl) * LS + pad16(z), spec + f * fstride + z * plane + (long)ky * Hx + kx0 + xl);
            }
        }
        if (nyq)
            for (int t = threadIdx.x; t < nf * N; t += blockDim.x) {
                const int f = t / N, z = t % N;
                cp_async<sizeof(C)>(buf + (nf * TX + f) * LS + pad16(z), spec + f * fstride + z * plane + (long)ky * Hx + N / 2);
            }
        cp_async_wait_all();
        __syncthreads();
    }
    if (mode == Z_FWD_GAMMA_INV || mode == Z_FWD_RESID) {
        const bool apply = mode == Z_FWD_GAMMA_INV;
        T acc = (T)0;   // per-thread sum in the field precision; block and global sums in FP64
        // one frequency: its six field values at p0 + f * fstep in the slab
        auto point = [&](int kz, int kx, C *p0, int fstep) {
            C s6[6];
            for (int f = 0; f < 6; ++f) s6[f] = p0[f * fstep];
            if (kx == 0 && ky == 0 && kz == 0 && mean6 != nullptr) {
                const double inv = 1.0 / ((double)N * N * N);
                for (int f = 0; f < 6; ++f) mean6[f] = (double)s6[f].x * inv;
            }
            const bool partner = !(kx == 0 || kx == (N >> 1));
            gamma_point<C, T>(s6, kx, ky, kz, N, lam0, mu0, acc, partner, apply);
            if (apply)
                for (int f = 0; f < 6; ++f) p0[f * fstep] = s6[f];
        };
        if constexpr (walk) {   // the same points per thread, in the same order, as the loop below
            C *pb = buf + wxl * LS + pad16(wz);
#pragma unroll
            for (int k = 0; k < KZ; ++k) point(wz + k * DZ, kx0 + wxl, pb + k * (DZ + DZ / 16), TX * LS);
            if (nyq)
                for (int t = threadIdx.x; t < N; t += blockDim.x) point(t, N / 2, buf + nf * TX * LS + pad16(t), LS);
        } else {
            const int npts = (TX + (nyq ? 1 : 0)) * N;
            for (int t = threadIdx.x; t < npts; t += blockDim.x) {
                const bool reg = t < TX * N;
                int zr = 0, xr = 0;
                if (reg) slab_item<N, TX>(t, zr, xr);
                const int kz = reg ? zr : t - TX * N;
                const int kx = reg ? kx0 + xr : N / 2;
                const int l0 = reg ? xr : nf * TX, ls = reg ? TX : 1;   // line of field f: l0 + f*ls
                point(kz, kx, buf + l0 * LS + pad16(kz), ls * LS);
            }
        }
        __syncthreads();
        const double tot = block_sum((double)acc, red);
        if (threadIdx.x == 0 && partials != nullptr) partials[blockIdx.x] = tot;
    }
    const bool inv = mode == Z_INV || mode == Z_FWD_GAMMA_INV;
    if constexpr (Shape<N>::R2 > 1) {
        if (inv) {
            bfft_pass1<N, true, MI>(buf, nlines);
            // the inverse transform's pass 2 stored straight to HBM: item (line, j < 16) transforms slots j + 16 r
            // as bfft_pass2 and stores elements j + 16 r
            constexpr int R2 = Shape<N>::R2;
            const int nit = nlines * 16;
            for (int it = threadIdx.x; it < nit; it += blockDim.x) {
                int l, j;
                C *g = hbm_item(it, 16, l, j);
                const C *line = buf + l * LS + j;
                C u[R2];
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    C a = line[17 * r];
                    if (r > 0) {
                        C w = tw[16 * r + j];
                        w.y = -w.y;
                        a = cmul(a, w);
                    }
                    u[r] = a;
                }
                dft_reg<R2, true>(u);
#pragma unroll
                for (int r = 0; r < R2; ++r) g[(long)(j + 16 * r) * plane] = u[r];
            }
        }
    } else if (inv) {
        block_fft<N, true, MI>(buf, nlines, tw);
    }
    if (!inv || Shape<N>::R2 == 1) {   // the slab from shared memory
        if constexpr (walk) {
            const C *sb = buf + wxl * LS + pad16(wz);
            C *gb = spec + (long)wz * plane + (long)ky * Hx + kx0 + wxl;
            for (int f = 0; f < nf; ++f) {
#pragma unroll
                for (int k = 0; k < KZ; ++k) gb[f * fstride + (long)k * DZ * plane] = sb[f * TX * LS + k * (DZ + DZ / 16)];
            }
        } else {
            for (int t = threadIdx.x; t < nf * TX * N; t += blockDim.x) {
                const int f = t / (TX * N), r = t % (TX * N);
                int z, xl;
                slab_item<N, TX>(r, z, xl);
                spec[f * fstride + z * plane + (long)ky * Hx + kx0 + xl] = buf[(f * TX + xl) * LS + pad16(z)];
            }
        }
        if (nyq)
            for (int t = threadIdx.x; t < nf * N; t += blockDim.x) {
                const int f = t / N, z = t % N;
                spec[f * fstride + z * plane + (long)ky * Hx + N / 2] = buf[(nf * TX + f) * LS + pad16(z)];
            }
    }
    if (zc.ctl != nullptr) {   // the last block to finish runs the fixed-point control (fpctl.cuh)
        __shared__ int last;
        __threadfence();       // this block's partial sum and spectrum are visible to the others
        __syncthreads();
        if (threadIdx.x == 0) last = atomicAdd(&zc.ctl->ticket, 1u) == gridDim.x - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
        fp_control_block<T>(zc, partials, gridDim.x, spec, fstride, N);
        if (threadIdx.x == 0) zc.ctl->ticket = 0u;
    }
}

template <typename T, int N> size_t smem_x() { return sizeof(typename CT<T>::type) * (N + (size_t)rowpairs<N>() * Shape<N>::LS); }
template <typename T, int N> size_t smem_y() { return sizeof(typename CT<T>::type) * (N + (size_t)(tx_y<N, T>() + 1) * Shape<N>::LS); }
template <typename T, int N> size_t smem_z(int nf) {
    return sizeof(typename CT<T>::type) * (N + (size_t)nf * (tx_z<N, T>() + 1) * Shape<N>::LS);
}

template <typename K> cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int N> cudaError_t x_r2c_n(const T *in, void *spec, int nfields, cudaStream_t s, const int *skip) {
    using C = typename CT<T>::type;
    const long npairs = (long)nfields * N * N / 2;
    const int blocks = (int)((npairs + rowpairs<N>() - 1) / rowpairs<N>());
    const size_t sm = smem_x<T, N>();
    cudaError_t e = allow_smem(k_fft_x_r2c<T, N>, sm);
    if (e != cudaSuccess) return e;
    return launch_k(skip != nullptr, k_fft_x_r2c<T, N>, dim3(blocks), dim3(kThreads), sm, s, in, (C *)spec, npairs, skip);
}

template <typename T, int N>
cudaError_t x_c2r_n(const void *spec, T *out, int nfields, T scale, const double *add6, cudaStream_t s, const T *base,
                    const int *skip) {
    using C = typename CT<T>::type;
    const long npairs = (long)nfields * N * N / 2;
    constexpr int RP = rowpairs_c2r<N>();
    const int blocks = (int)((npairs + RP - 1) / RP);
    const size_t sm = sizeof(C) * (N + (size_t)RP * Shape<N>::LS + 2 * (size_t)RP * (N / 2 + 1)) +
                      sizeof(T) * 2 * (size_t)RP * N;
    cudaError_t e = allow_smem(k_fft_x_c2r<T, N>, sm);
    if (e != cudaSuccess) return e;
    T a[6] = {0, 0, 0, 0, 0, 0};   // rounded to the field precision here, not once per element on the device
    if (add6)
        for (int i = 0; i < 6; ++i) a[i] = (T)add6[i];
    const int has_add = add6 != nullptr;
    return launch_k(skip != nullptr, k_fft_x_c2r<T, N>, dim3(blocks), dim3(kThreads), sm, s, (const C *)spec, out, npairs,
                    scale, has_add, a[0], a[1], a[2], a[3], a[4], a[5], base, skip);
}

template <typename T, int N> cudaError_t y_n(void *spec, int nfields, int inverse, cudaStream_t s, const int *skip) {
    using C = typename CT<T>::type;
    constexpr int TX = tx_y<N, T>();
    const int blocks = nfields * N * ((N / 2) / TX);
    const size_t sm = smem_y<T, N>();
    cudaError_t e = inverse ? allow_smem(k_fft_y<T, N, true>, sm) : allow_smem(k_fft_y<T, N, false>, sm);
    if (e != cudaSuccess) return e;
    if (inverse) return launch_k(skip != nullptr, k_fft_y<T, N, true>, dim3(blocks), dim3(y_threads<N, T>()), sm, s, (C *)spec, skip);
    return launch_k(skip != nullptr, k_fft_y<T, N, false>, dim3(blocks), dim3(y_threads<N, T>()), sm, s, (C *)spec, skip);
}

// x and y passes of the forward transform: one fused launch where the plane fits (xy_fused), else the two passes
template <typename T, int N> cudaError_t xy_r2c_n(const T *in, void *spec, int nfields, cudaStream_t s, const int *skip) {
    if constexpr (xy_fused<T, N>()) {
        using C = typename CT<T>::type;
        constexpr size_t sm = smem_xy<T, N>();
        cudaError_t e = allow_smem(k_fft_xy_r2c<T, N>, sm);
        if (e != cudaSuccess) return e;
        return launch_k(skip != nullptr, k_fft_xy_r2c<T, N>, dim3(nfields * N), dim3(xy_threads<N>()), sm, s, in,
                        (C *)spec, skip);
    } else {
        cudaError_t e = x_r2c_n<T, N>(in, spec, nfields, s, skip);
        if (e != cudaSuccess) return e;
        return y_n<T, N>(spec, nfields, 0, s, skip);
    }
}

template <typename T, int N>
cudaError_t xy_c2r_n(const void *spec, T *out, int nfields, T scale, const double *add6, cudaStream_t s, const T *base,
                     const int *skip) {
    if constexpr (xy_fused<T, N>()) {
        using C = typename CT<T>::type;
        constexpr size_t sm = smem_xy<T, N>();
        cudaError_t e = allow_smem(k_fft_xy_c2r<T, N>, sm);
        if (e != cudaSuccess) return e;
        T a[6] = {0, 0, 0, 0, 0, 0};   // rounded to the field precision here, as in the x pass
        if (add6)
            for (int i = 0; i < 6; ++i) a[i] = (T)add6[i];
        const int has_add = add6 != nullptr;
        return launch_k(skip != nullptr, k_fft_xy_c2r<T, N>, dim3(nfields * N), dim3(xy_threads<N>()), sm, s,
                        (const C *)spec, out, scale, has_add, a[0], a[1], a[2], a[3], a[4], a[5], base, skip);
    } else {
        cudaError_t e = y_n<T, N>(const_cast<void *>(spec), nfields, 1, s, skip);
        if (e != cudaSuccess) return e;
        return x_c2r_n<T, N>(spec, out, nfields, scale, add6, s, base, skip);
    }
}

template <typename T, int N>
cudaError_t z_n(void *spec, int nfields, int mode, double lam0, double mu0, double *partials, double *mean6,
                cudaStream_t s, const int *skip, const ZCtl *zcp) {
    using C = typename CT<T>::type;
    constexpr int TX = tx_z<N, T>();
    const int blocks = N * ((N / 2) / TX);
    const size_t sm = smem_z<T, N>(nfields);
    cudaError_t e = allow_smem(k_fft_z<T, N>, smem_z<T, N>(6));
    if (e != cudaSuccess) return e;
    ZCtl zc{};
    if (zcp != nullptr) zc = *zcp;
    return launch_k(skip != nullptr, k_fft_z<T, N>, dim3(blocks), dim3(z_threads<N, T>()), sm, s, (C *)spec, nfields, mode,
                    (T)lam0, (T)mu0, partials, mean6, skip, zc);
}

#define EVP_DISPATCH(N_, CALL)                             \
    switch (N_) {                                          \
        case 4: { constexpr int NN = 4; return CALL; }     \
        case 8: { constexpr int NN = 8; return CALL; }     \
        case 16: { constexpr int NN = 16; return CALL; }   \
        case 32: { constexpr int NN = 32; return CALL; }   \
        case 64: { constexpr int NN = 64; return CALL; }   \
        case 128: { constexpr int NN = 128; return CALL; } \
        case 256: { constexpr int NN = 256; return CALL; } \
        default: return cudaErrorInvalidValue;             \
    }

}  // namespace

int fft_z_blocks(int n, int is_double) {
    const int TX0 = is_double ? 4 : 8;
    const int TX = TX0 < n / 2 ? TX0 : n / 2;
    return n * ((n / 2) / TX);
}

int fft_xy_fused(int n, int is_double) {
    if (is_double) {
        EVP_DISPATCH(n, (int)(xy_fused<double, NN>()))
    }
    EVP_DISPATCH(n, (int)(xy_fused<float, NN>()))
}

template <typename T>
cudaError_t fft_xy_r2c(const T *in, void *spec, int n, int nfields, cudaStream_t s, const int *skip) {
    EVP_DISPATCH(n, (xy_r2c_n<T, NN>(in, spec, nfields, s, skip)))
}

template <typename T>
cudaError_t fft_xy_c2r(const void *spec, T *out, int n, int nfields, T scale, const double *add6, cudaStream_t s,
                       const T *base, const int *skip) {
    // the same contract as the x pass (whole rows in 16-byte chunks where the passes run separately)
    if (((uintptr_t)spec | (uintptr_t)out | (uintptr_t)base) & 15) return cudaErrorInvalidValue;
    EVP_DISPATCH(n, (xy_c2r_n<T, NN>(spec, out, nfields, scale, add6, s, base, skip)))
}

template <typename T>
cudaError_t fft_x_r2c(const T *in, void *spec, int n, int nfields, cudaStream_t s, const int *skip) {
    EVP_DISPATCH(n, (x_r2c_n<T, NN>(in, spec, nfields, s, skip)))
}

template <typename T>
cudaError_t fft_x_c2r(const void *spec, T *out, int n, int nfields, T scale, const double *add6, cudaStream_t s,
                      const T *base, const int *skip) {
    // the pass copies whole rows in 16-byte chunks
    if (((uintptr_t)spec | (uintptr_t)out | (uintptr_t)base) & 15) return cudaErrorInvalidValue;
    EVP_DISPATCH(n, (x_c2r_n<T, NN>(spec, out, nfields, scale, add6, s, base, skip)))
}

template <typename T> cudaError_t fft_y(void *spec, int n, int nfields, int inverse, cudaStream_t s, const int *skip) {
    EVP_DISPATCH(n, (y_n<T, NN>(spec, nfields, inverse, s, skip)))
}

template <typename T>
cudaError_t fft_z(void *spec, int n, int nfields, int mode, double lam0, double mu0, double *partials, double *mean6,
                  cudaStream_t s, const int *skip, const ZCtl *zc) {
    if ((mode == Z_FWD_GAMMA_INV || mode == Z_FWD_RESID) && nfields != 6) return cudaErrorInvalidValue;
    if (zc != nullptr && (mode != Z_FWD_GAMMA_INV || partials == nullptr)) return cudaErrorInvalidValue;
    EVP_DISPATCH(n, (z_n<T, NN>(spec, nfields, mode, lam0, mu0, partials, mean6, s, skip, zc)))
}

#define EVP_FFT_INST(T)                                                                                            \
    template cudaError_t fft_x_r2c<T>(const T *, void *, int, int, cudaStream_t, const int *);                     \
    template cudaError_t fft_x_c2r<T>(const void *, T *, int, int, T, const double *, cudaStream_t, const T *,     \
                                      const int *);                                                                \
    template cudaError_t fft_y<T>(void *, int, int, int, cudaStream_t, const int *);                               \
    template cudaError_t fft_xy_r2c<T>(const T *, void *, int, int, cudaStream_t, const int *);                    \
    template cudaError_t fft_xy_c2r<T>(const void *, T *, int, int, T, const double *, cudaStream_t, const T *,    \
                                       const int *);                                                               \
    template cudaError_t fft_z<T>(void *, int, int, int, double, double, double *, double *, cudaStream_t,         \
                                  const int *, const ZCtl *);
EVP_FFT_INST(float)
EVP_FFT_INST(double)
#undef EVP_FFT_INST

}  // namespace evp
